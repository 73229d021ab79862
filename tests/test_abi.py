"""CPU-side checks of the C ABI: the library builds, loads, and exports every
entry point that include/lsg.h declares; host-side argument validation.
No kernel runs here (there is no GPU on this side)."""
import ctypes
import os
import re

from paper_2005_02704_gb300 import lsg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(lsg_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("lsg_create", "lsg_destroy", "lsg_segment", "lsg_label_from_mask", "lsg_batch_plan",
                 "lsg_batch_run", "lsg_autotune", "lsg_plan_destroy", "lsg_get_error", "lsg_status_str",
                 "lsg_default_params"):
        assert want in names


def test_library_exports_every_declared_symbol():
    lib = lsg.load()
    for name in sorted(declared_functions()):
        assert hasattr(lib, name), name


def test_struct_layouts_match_the_header():
    # offsets follow from the header's field order and natural alignment
    assert ctypes.sizeof(lsg.lsg_scan) == 40
    assert lsg.lsg_scan.xyzr.offset == 24
    assert ctypes.sizeof(lsg.lsg_params) == 44
    assert lsg.lsg_params.comp.offset == 28
    assert ctypes.sizeof(lsg.lsg_out) == 32


def test_defaults_and_status_strings():
    p = lsg.lsg_default_params()
    assert p.subsample == 1 and p.wrap == 1 and p.predicate == lsg.LSG_PRED_ANGLE
    assert abs(p.angle_rad - 0.17453292) < 1e-6
    assert abs(p.jump_rel_h - 0.1) < 1e-7 and p.jump_rel_v == 1.0
    assert lsg.lsg_status_str(lsg.LSG_OK) == "ok"
    assert lsg.lsg_status_str(lsg.LSG_E_BUDGET) == "memory budget exceeded"


def test_null_arguments_are_rejected_without_a_device():
    lib = lsg.load()
    assert lib.lsg_segment(None, None, None, None, None) == lsg.LSG_E_ARG
    assert lib.lsg_destroy(None) == lsg.LSG_E_ARG
    assert lib.lsg_batch_run(None, None) == lsg.LSG_E_ARG
    assert lib.lsg_get_error(None) == lsg.LSG_E_ARG
    assert lib.lsg_plan_launches(None) == -1 and lib.lsg_plan_tile(None) == -1
    assert lib.lsg_selftest_wait_timeout(None) == lsg.LSG_E_ARG
    h = ctypes.c_void_p()
    # no CUDA device on this side: creating a context must fail cleanly
    import torch
    if not torch.cuda.is_available():
        assert lib.lsg_create(0, 0, ctypes.byref(h)) == lsg.LSG_E_ARG
        assert h.value is None


def test_spin_entry_points_reject_null_handles():
    lib = lsg.load()
    assert lib.lsg_spin_begin(None, None, None, None, None, None) == lsg.LSG_E_ARG
    assert lib.lsg_spin_push(None, 0, None) == lsg.LSG_E_ARG
    assert lib.lsg_spin_finish(None, None) == lsg.LSG_E_ARG
    assert lib.lsg_spin_destroy(None) == lsg.LSG_E_ARG

"""ctypes front end of the FP64 oracle (``lsg_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Arrays in, arrays out;
the arithmetic is all in the C file, which follows Sec. 2 and Algorithm 1 of
Mukherjee et al. (PReMI 2019) step by step.
"""
from __future__ import annotations

import ctypes
import math
import os
import shutil
import subprocess
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lsg_oracle.c")
_LIB = os.path.join(_HERE, "liblsg_oracle.so")

PRED_ANGLE = 0
PRED_COMPONENT = 1

BIT_R, BIT_D, BIT_G = 0x01, 0x02, 0x04
BIT_HR, BIT_HD, BIT_HG = 0x08, 0x10, 0x20
BIT_VALID, BIT_HASN = 0x40, 0x80


def build(force: bool = False) -> str:
    """Compile the oracle with plain gcc (-O2, no fused multiply-add contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler for the oracle")
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.run([cc, "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    _SRC, "-o", tmp, "-lm"], check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None
_P = ctypes.c_void_p


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        I, F, D = ctypes.c_int, ctypes.c_float, ctypes.c_double
        sig = {
            "oracle_ring_order": [I, _P, _P],
            "oracle_decode": [I, I, _P, _P, F, F, _P, _P, F, F, _P, _P, _P],
            "oracle_mesh": [I, I, I, I, _P, _P, F, F, _P],
            "oracle_neighbours": [I, I, I, I, _P, _P, _P],
            "oracle_normals": [I, I, I, I, F, _P, _P, _P, _P, _P, _P],
            "oracle_edge_mask": [I, I, I, I, I, D, _P, _P, _P, _P],
            "oracle_components": [I, I, I, I, _P, _P],
            "oracle_algorithm1": [I, I, I, I, _P, _P],
            "oracle_backfill": [I, I, I, I, _P, _P, _P],
            "oracle_segment": [I, I, _P, F, F, _P, _P, I, F, F, F, F, I, D, _P, I, _P, _P, _P, _P, _P,
                               _P, _P, _P, _P, _P],
            "oracle_label_from_mask": [I, I, I, I, _P, _P, _P, _P],
            "oracle_segment_stats": [I, I, I, _P, _P, _P, I, _P, _P, _P],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = I
        lib.oracle_angle.argtypes = [_P, _P]
        lib.oracle_angle.restype = D
        _lib = lib
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


@dataclass
class Params:
    """Segmentation parameters (same meaning as the C-ABI's lsg_params)."""
    subsample: int = 1
    r_min: float = 0.0
    r_max: float = 100.0
    jump_rel_h: float = 0.10
    jump_rel_v: float = 1.0
    predicate: int = PRED_ANGLE
    angle_rad: float = math.radians(10.0)
    comp: Sequence[float] = (0.2, 0.2, 0.2)
    wrap: int = 1


@dataclass
class Result:
    order: np.ndarray      # int32 [H]   sorted ring -> input row
    meshbits: np.ndarray   # uint8 [H, Ws]
    normals: np.ndarray    # float64 [H, Ws, 3]
    labels: np.ndarray     # int32 [H, W]
    nseg: int
    kappa: np.ndarray      # float64 [H, Ws]
    margin: np.ndarray     # float64 [H, Ws, 3]
    vlabel: np.ndarray     # int32 [H, Ws]
    snorm: np.ndarray      # float64 [H, Ws]  |sum_k w_k V_k x V_k+1|
    ntri: np.ndarray       # int32 [H, Ws]    counted triangles


def ws_of(W: int, s: int) -> int:
    return (W + s - 1) // s


def ring_order(elev) -> np.ndarray:
    e = _c(elev, np.float32)
    order = np.zeros(len(e), dtype=np.int32)
    if _load().oracle_ring_order(len(e), _ptr(e), _ptr(order)) != 0:
        raise ValueError("NaN elevation")
    return order


def segment(elev, az0: float, daz: float, xyzr: Optional[np.ndarray], p: Params,
            range_: Optional[np.ndarray] = None) -> Result:
    """Every step of the path on one scan.  ``xyzr`` float32 [H, W, 4] in input
    ring order, or None with ``range_`` float32 [H, W] (range-only decode)."""
    lib = _load()
    e = _c(elev, np.float32)
    H = len(e)
    if xyzr is not None:
        xyzr = _c(xyzr, np.float32)
        W = xyzr.shape[1] if H else 0
    else:
        range_ = _c(range_, np.float32)
        W = range_.shape[1] if H else 0
    s = int(p.subsample)
    Ws = ws_of(W, s) if W else 0
    order = np.zeros(H, dtype=np.int32)
    mb = np.zeros((H, Ws), dtype=np.uint8)
    nrm = np.zeros((H, Ws, 3), dtype=np.float64)
    labels = np.full((H, W), -1, dtype=np.int32)
    kappa = np.zeros((H, Ws), dtype=np.float64)
    margin = np.zeros((H, Ws, 3), dtype=np.float64)
    vlabel = np.full((H, Ws), -1, dtype=np.int32)
    snorm = np.zeros((H, Ws), dtype=np.float64)
    ntri = np.zeros((H, Ws), dtype=np.int32)
    nseg = np.zeros(1, dtype=np.int32)
    comp = _c(p.comp, np.float64)
    rc = lib.oracle_segment(H, W, _ptr(e), float(az0), float(daz), _ptr(xyzr), _ptr(range_), s,
                            float(p.r_min), float(p.r_max), float(p.jump_rel_h), float(p.jump_rel_v),
                            int(p.predicate), float(p.angle_rad), _ptr(comp), int(p.wrap), _ptr(order),
                            _ptr(mb), _ptr(nrm), _ptr(labels), _ptr(nseg), _ptr(kappa), _ptr(margin),
                            _ptr(vlabel), _ptr(snorm), _ptr(ntri))
    if rc != 0:
        raise ValueError(f"oracle_segment failed: {rc}")
    return Result(order, mb, nrm, labels, int(nseg[0]), kappa, margin, vlabel, snorm, ntri)


def segment_scan(scan, p: Params, range_only: bool = False) -> Result:
    """Convenience wrapper for a ``lidarsim.Scan``."""
    if range_only:
        return segment(scan.elev, scan.az0, scan.daz, None, p, scan.range)
    return segment(scan.elev, scan.az0, scan.daz, scan.xyzr, p)


# ---- single steps (used by the oracle's own pin tests) --------------------
def decode(elev, az0, daz, xyzr, range_, r_min, r_max):
    lib = _load()
    e = _c(elev, np.float32)
    H = len(e)
    src = xyzr if xyzr is not None else range_
    W = src.shape[1]
    order = ring_order(e)
    rs = np.zeros((H, W), np.float32)
    xyz = np.zeros((H, W, 3), np.float64)
    valid = np.zeros((H, W), np.uint8)
    lib.oracle_decode(H, W, _ptr(order), _ptr(e), float(az0), float(daz),
                      _ptr(None if xyzr is None else _c(xyzr, np.float32)),
                      _ptr(None if range_ is None else _c(range_, np.float32)),
                      float(r_min), float(r_max), _ptr(rs), _ptr(xyz), _ptr(valid))
    return order, rs, xyz, valid


def mesh(rs, valid, s, wrap, jump_h, jump_v):
    lib = _load()
    rs = _c(rs, np.float32)
    valid = _c(valid, np.uint8)
    H, W = rs.shape
    mb = np.zeros((H, ws_of(W, s)), np.uint8)
    lib.oracle_mesh(H, W, s, wrap, _ptr(rs), _ptr(valid), float(jump_h), float(jump_v), _ptr(mb))
    return mb


def neighbours(mb, W, s, wrap):
    lib = _load()
    mb = _c(mb, np.uint8)
    H, Ws = mb.shape
    nbr = np.zeros((H, Ws, 6), np.int32)
    cnt = np.zeros((H, Ws), np.int32)
    lib.oracle_neighbours(H, W, s, wrap, _ptr(mb), _ptr(nbr), _ptr(cnt))
    return nbr, cnt


def normals(xyz, mb, W, s, wrap, daz):
    lib = _load()
    xyz = _c(xyz, np.float64)
    mb = _c(mb, np.uint8).copy()
    H, Ws = mb.shape
    nrm = np.zeros((H, Ws, 3), np.float64)
    kappa = np.zeros((H, Ws), np.float64)
    lib.oracle_normals(H, W, s, wrap, float(daz), _ptr(xyz), _ptr(mb), _ptr(nrm), _ptr(kappa), None, None)
    return mb, nrm, kappa


def edge_mask(normal, mb, W, s, wrap, pred, angle_t, comp=(0.2, 0.2, 0.2)):
    lib = _load()
    normal = _c(normal, np.float64)
    mb = _c(mb, np.uint8).copy()
    H, Ws = mb.shape
    margin = np.zeros((H, Ws, 3), np.float64)
    compa = _c(comp, np.float64)
    lib.oracle_edge_mask(H, W, s, wrap, int(pred), float(angle_t), _ptr(compa), _ptr(normal), _ptr(mb),
                         _ptr(margin))
    return mb, margin


def components(mb, W, s, wrap):
    lib = _load()
    mb = _c(mb, np.uint8)
    H, Ws = mb.shape
    vl = np.full((H, Ws), -1, np.int32)
    n = lib.oracle_components(H, W, s, wrap, _ptr(mb), _ptr(vl))
    return vl, n


def algorithm1(mb, W, s, wrap):
    lib = _load()
    mb = _c(mb, np.uint8)
    H, Ws = mb.shape
    L = np.zeros((H, Ws), np.int32)
    n = lib.oracle_algorithm1(H, W, s, wrap, _ptr(mb), _ptr(L))
    return L, n


def backfill(valid, vlabel, W, s, wrap):
    lib = _load()
    valid = _c(valid, np.uint8)
    vlabel = _c(vlabel, np.int32)
    H = valid.shape[0]
    out = np.full((H, W), -1, np.int32)
    lib.oracle_backfill(H, W, s, wrap, _ptr(valid), _ptr(vlabel), _ptr(out))
    return out


def label_from_mask(mb, valid, W, s, wrap):
    """Labels and segment count from a given mesh byte array (edge mask taken
    as given) and per-point validity [H, W] in sorted ring order."""
    lib = _load()
    mb = _c(mb, np.uint8)
    valid = _c(valid, np.uint8)
    H = mb.shape[0]
    labels = np.full((H, W), -1, np.int32)
    nseg = np.zeros(1, np.int32)
    rc = lib.oracle_label_from_mask(H, W, s, wrap, _ptr(mb), _ptr(valid), _ptr(labels), _ptr(nseg))
    if rc != 0:
        raise RuntimeError("oracle_label_from_mask failed")
    return labels, int(nseg[0])


def segment_stats(labels, min_points, W=None, s=1, normals=None, meshbits=None):
    """Sizes of the segments, optional normal sums, and labels with the
    segments of fewer than min_points points removed (Sec. 2, last
    paragraph).  Returns (labels_out, sizes, nsum or None, kept)."""
    lib = _load()
    labels = _c(labels, np.int32)
    H, W_ = labels.shape
    out = np.empty_like(labels)
    sizes = np.zeros(H * W_, np.int32)
    nsum = np.zeros((H * W_, 3), np.float64) if normals is not None else None
    nrm = _c(normals, np.float64) if normals is not None else None
    mb = _c(meshbits, np.uint8) if meshbits is not None else None
    kept = lib.oracle_segment_stats(H, W_, int(s), _ptr(labels), _ptr(nrm), _ptr(mb), int(min_points), _ptr(out),
                                    _ptr(sizes), _ptr(nsum))
    return out, sizes, nsum, kept


def angle(a, b) -> float:
    a = _c(a, np.float64)
    b = _c(b, np.float64)
    return _load().oracle_angle(_ptr(a), _ptr(b))


__all__ = ["Params", "Result", "segment", "segment_scan", "ring_order", "decode", "mesh", "neighbours",
           "normals", "edge_mask", "components", "algorithm1", "backfill", "label_from_mask", "angle",
           "segment_stats",
           "ws_of", "build", "PRED_ANGLE", "PRED_COMPONENT", "BIT_R", "BIT_D", "BIT_G", "BIT_HR",
           "BIT_HD", "BIT_HG", "BIT_VALID", "BIT_HASN"]

"""Python binding of the C ABI in ``include/lsg.h`` (ctypes; argument
marshalling only).

The functions keep the C names (``lsg_segment``, ``lsg_batch_plan``, ...) and
take raw device pointers; ``Context`` is a thin convenience layer that
allocates outputs with PyTorch (device memory and streams only) and calls the
same entry points.  Every step of the path runs in the library's CUDA
kernels; there is no CPU fallback, and ``load()`` raises when the library
cannot be built or loaded.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass
from typing import List, Optional, Sequence

from . import _build

LSG_OK, LSG_E_ARG, LSG_E_SHAPE, LSG_E_OOM, LSG_E_BUDGET, LSG_E_CUDA, LSG_E_TIMEOUT, LSG_E_DEVICE = range(8)
LSG_PRED_ANGLE, LSG_PRED_COMPONENT = 0, 1
LSG_TILE_AUTO = -1
TILES = {"16x240": 0, "32x120": 1, "32x240": 2, "32x480": 3, "64x240": 4, "16x120": 5, "8x120": 6, "4x120": 7,
         "2x120": 8}
LSG_TILE_COUNT = len(TILES)

BIT_R, BIT_D, BIT_G = 0x01, 0x02, 0x04
BIT_HR, BIT_HD, BIT_HG = 0x08, 0x10, 0x20
BIT_VALID, BIT_HASN = 0x40, 0x80


class lsg_scan(ctypes.Structure):
    _fields_ = [("rings", ctypes.c_int32), ("cols", ctypes.c_int32), ("elevation", ctypes.c_void_p),
                ("azimuth0", ctypes.c_float), ("azimuth_step", ctypes.c_float),
                ("xyzr", ctypes.c_void_p), ("range", ctypes.c_void_p)]


class lsg_params(ctypes.Structure):
    _fields_ = [("subsample", ctypes.c_int32), ("r_min", ctypes.c_float), ("r_max", ctypes.c_float),
                ("jump_rel_h", ctypes.c_float), ("jump_rel_v", ctypes.c_float),
                ("predicate", ctypes.c_int32), ("angle_rad", ctypes.c_float),
                ("comp", ctypes.c_float * 3), ("wrap", ctypes.c_int32)]


class lsg_out(ctypes.Structure):
    _fields_ = [("meshbits", ctypes.c_void_p), ("normals", ctypes.c_void_p),
                ("labels", ctypes.c_void_p), ("nseg", ctypes.c_void_p)]


class lsg_host_io(ctypes.Structure):
    _fields_ = [("xyzr", ctypes.c_void_p), ("elevation", ctypes.c_void_p), ("labels", ctypes.c_void_p),
                ("nseg", ctypes.c_void_p), ("meshbits", ctypes.c_void_p), ("normals", ctypes.c_void_p)]


class lsg_raycast_spec(ctypes.Structure):
    _fields_ = [("rings", ctypes.c_int32), ("cols", ctypes.c_int32), ("elevation", ctypes.c_void_p),
                ("azimuth0", ctypes.c_float), ("azimuth_step", ctypes.c_float), ("nprims", ctypes.c_int32),
                ("prims", ctypes.c_void_p), ("sigma", ctypes.c_double), ("p_drop", ctypes.c_double),
                ("r_max", ctypes.c_double), ("seed", ctypes.c_uint64)]


LSG_RAYCAST_MAX_PRIMS = 256
LSG_PRIM_PLANE, LSG_PRIM_BOX, LSG_PRIM_CYL = 0, 1, 2


class LsgError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {lsg_status_str(status)} ({status})")
        self.status = status


_lib = None
_P = ctypes.c_void_p


def load(build: bool = True):
    """Load ``liblsg.so`` (building it in-tree first when it is stale)."""
    global _lib
    if _lib is None:
        path = _build.build() if build else _build.LIB
        lib = ctypes.CDLL(path)
        I32 = ctypes.c_int32
        sig = {
            "lsg_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(_P)]),
            "lsg_destroy": (ctypes.c_int, [_P]),
            "lsg_set_tile": (ctypes.c_int, [_P, ctypes.c_int]),
            "lsg_segment": (ctypes.c_int, [_P, ctypes.POINTER(lsg_scan), ctypes.POINTER(lsg_params),
                                           ctypes.POINTER(lsg_out), _P]),
            "lsg_label_from_mask": (ctypes.c_int, [_P, I32, I32, I32, I32, _P, _P, _P, _P, _P]),
            "lsg_batch_plan": (ctypes.c_int, [_P, I32, ctypes.POINTER(lsg_scan), ctypes.POINTER(lsg_params),
                                              ctypes.POINTER(lsg_out), ctypes.c_int, ctypes.POINTER(_P)]),
            "lsg_batch_run": (ctypes.c_int, [_P, _P]),
            "lsg_batch_plan_io": (ctypes.c_int, [_P, I32, ctypes.POINTER(lsg_scan), ctypes.POINTER(lsg_params),
                                                 ctypes.POINTER(lsg_out), ctypes.POINTER(lsg_host_io), I32,
                                                 ctypes.c_int, ctypes.POINTER(_P)]),
            "lsg_plan_io_bytes": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_size_t),
                                                 ctypes.POINTER(ctypes.c_size_t)]),
            "lsg_batch_launch": (ctypes.c_int, [_P, I32, ctypes.POINTER(lsg_scan), ctypes.POINTER(lsg_params),
                                                ctypes.POINTER(lsg_out), _P]),
            "lsg_batch_launch_io": (ctypes.c_int, [_P, I32, ctypes.POINTER(lsg_scan), ctypes.POINTER(lsg_params),
                                                   ctypes.POINTER(lsg_out), ctypes.POINTER(lsg_host_io), _P]),
            "lsg_reserve": (ctypes.c_int, [_P, ctypes.c_size_t, I32, I32]),
            "lsg_autotune": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_float)]),
            "lsg_plan_tile": (ctypes.c_int, [_P]),
            "lsg_plan_set_fused": (ctypes.c_int, [_P, ctypes.c_int]),
            "lsg_plan_fused": (ctypes.c_int, [_P]),
            "lsg_plan_launches": (ctypes.c_int, [_P]),
            "lsg_plan_phase_times": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float)]),
            "lsg_plan_destroy": (ctypes.c_int, [_P]),
            "lsg_get_error": (ctypes.c_int, [_P]),
            "lsg_memory_used": (ctypes.c_size_t, [_P]),
            "lsg_selftest_wait_timeout": (ctypes.c_int, [_P]),
            "lsg_segment_stats": (ctypes.c_int, [_P, I32, I32, I32, I32, _P, _P, _P, _P, _P, _P, _P]),
            "lsg_segment_noalloc": (ctypes.c_int, [ctypes.POINTER(lsg_scan), ctypes.POINTER(lsg_params),
                                                   ctypes.POINTER(lsg_out), _P]),
            "lsg_noalloc_get_error": (ctypes.c_int, [_P]),
            "lsg_raycast": (ctypes.c_int, [ctypes.POINTER(lsg_raycast_spec), _P, _P, _P]),
            "lsg_spin_begin": (ctypes.c_int, [_P, ctypes.POINTER(lsg_scan), ctypes.POINTER(lsg_params),
                                              ctypes.POINTER(lsg_out), ctypes.POINTER(_P), _P]),
            "lsg_spin_push": (ctypes.c_int, [_P, I32, _P]),
            "lsg_spin_finish": (ctypes.c_int, [_P, _P]),
            "lsg_spin_destroy": (ctypes.c_int, [_P]),
            "lsg_default_params": (None, [ctypes.POINTER(lsg_params)]),
            "lsg_status_str": (ctypes.c_char_p, [ctypes.c_int]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


# ---- the C entry points, same names -------------------------------------
def lsg_status_str(status: int) -> str:
    return load().lsg_status_str(status).decode()


def _check(status: int, what: str):
    if status != LSG_OK:
        raise LsgError(status, what)


def lsg_default_params() -> lsg_params:
    p = lsg_params()
    load().lsg_default_params(ctypes.byref(p))
    return p


def lsg_create(device: int = 0, budget_bytes: int = 0) -> int:
    h = _P()
    _check(load().lsg_create(device, budget_bytes, ctypes.byref(h)), "lsg_create")
    return h.value


def lsg_destroy(ctx: int) -> None:
    _check(load().lsg_destroy(ctx), "lsg_destroy")


def lsg_set_tile(ctx: int, tile: int) -> None:
    _check(load().lsg_set_tile(ctx, tile), "lsg_set_tile")


def lsg_segment(ctx: int, scan: lsg_scan, params: lsg_params, out: lsg_out, stream: int = 0) -> int:
    """Returns the status code (callers that want exceptions use Context)."""
    return load().lsg_segment(ctx, ctypes.byref(scan), ctypes.byref(params), ctypes.byref(out), stream or None)


def lsg_label_from_mask(ctx: int, H: int, W: int, s: int, wrap: int, meshbits: int, valid: int,
                        labels: int, nseg: int, stream: int = 0) -> int:
    return load().lsg_label_from_mask(ctx, H, W, s, wrap, meshbits or None, valid or None, labels or None,
                                      nseg or None, stream or None)


def lsg_batch_plan(ctx: int, scans: Sequence[lsg_scan], params: Sequence[lsg_params],
                   outs: Sequence[lsg_out], tile: int = LSG_TILE_AUTO) -> int:
    n = len(scans)
    sa = (lsg_scan * n)(*scans)
    pa = (lsg_params * n)(*params)
    oa = (lsg_out * n)(*outs)
    h = _P()
    _check(load().lsg_batch_plan(ctx, n, sa, pa, oa, tile, ctypes.byref(h)), "lsg_batch_plan")
    return h.value


def lsg_batch_plan_io(ctx: int, scans: Sequence[lsg_scan], params: Sequence[lsg_params],
                      outs: Sequence[lsg_out], io: Sequence[lsg_host_io], chunks: int,
                      tile: int = LSG_TILE_AUTO) -> int:
    n = len(scans)
    sa = (lsg_scan * n)(*scans)
    pa = (lsg_params * n)(*params)
    oa = (lsg_out * n)(*outs)
    ia = (lsg_host_io * n)(*io)
    h = _P()
    _check(load().lsg_batch_plan_io(ctx, n, sa, pa, oa, ia, int(chunks), tile, ctypes.byref(h)), "lsg_batch_plan_io")
    return h.value


def lsg_plan_io_bytes(plan: int):
    h2d, d2h = ctypes.c_size_t(), ctypes.c_size_t()
    _check(load().lsg_plan_io_bytes(plan, ctypes.byref(h2d), ctypes.byref(d2h)), "lsg_plan_io_bytes")
    return h2d.value, d2h.value


def lsg_batch_run(plan: int, stream: int = 0) -> int:
    return load().lsg_batch_run(plan, stream or None)


def lsg_batch_launch(ctx: int, scans, params, outs, stream: int = 0) -> int:
    """One pass over a changing set of scans (arrays of lsg_scan / lsg_params /
    lsg_out, or ctypes arrays of them).  Returns the status code."""
    n = len(scans)
    sa = scans if isinstance(scans, ctypes.Array) else (lsg_scan * n)(*scans)
    pa = params if isinstance(params, ctypes.Array) else (lsg_params * n)(*params)
    oa = outs if isinstance(outs, ctypes.Array) else (lsg_out * n)(*outs)
    return load().lsg_batch_launch(ctx, n, sa, pa, oa, stream or None)


def lsg_batch_launch_io(ctx: int, scans, params, outs, io, stream: int = 0) -> int:
    """lsg_batch_launch plus the host->device input and device->host result
    copies of each scan (sequences or ctypes arrays of lsg_scan / lsg_params /
    lsg_out / lsg_host_io).  Returns the status code."""
    n = len(scans)
    sa = scans if isinstance(scans, ctypes.Array) else (lsg_scan * n)(*scans)
    pa = params if isinstance(params, ctypes.Array) else (lsg_params * n)(*params)
    oa = outs if isinstance(outs, ctypes.Array) else (lsg_out * n)(*outs)
    ia = io if isinstance(io, ctypes.Array) else (lsg_host_io * n)(*io)
    return load().lsg_batch_launch_io(ctx, n, sa, pa, oa, ia, stream or None)


def lsg_reserve(ctx: int, workspace_bytes: int, max_scans: int, max_tiles: int) -> None:
    _check(load().lsg_reserve(ctx, workspace_bytes, max_scans, max_tiles), "lsg_reserve")


def scan_workspace_bytes(H: int, Ws: int) -> int:
    """Workspace of one scan inside a batch (four arrays, 256-byte aligned)."""
    up = lambda x: (x + 255) // 256 * 256
    return up(4 * H) + up(8 * H) + up(4 * H * Ws) + up(2 * H * ((Ws + 7) & ~7))


def lsg_autotune(plan: int, reps: int = 3, stream: int = 0):
    t = ctypes.c_int()
    ms = ctypes.c_float()
    _check(load().lsg_autotune(plan, reps, stream or None, ctypes.byref(t), ctypes.byref(ms)), "lsg_autotune")
    return t.value, ms.value


def lsg_plan_tile(plan: int) -> int:
    return load().lsg_plan_tile(plan)


def lsg_plan_set_fused(plan: int, schedule: int) -> None:
    """0 phased, 1 one persistent launch, 2 scan groups on overlapping branches."""
    _check(load().lsg_plan_set_fused(plan, int(schedule)), "lsg_plan_set_fused")


def lsg_plan_phase_times(plan: int):
    ms = (ctypes.c_float * 4)()
    _check(load().lsg_plan_phase_times(plan, ms), "lsg_plan_phase_times")
    return list(ms)


def lsg_plan_destroy(plan: int) -> None:
    _check(load().lsg_plan_destroy(plan), "lsg_plan_destroy")


def lsg_get_error(ctx: int) -> int:
    return load().lsg_get_error(ctx)


def lsg_memory_used(ctx: int) -> int:
    """Device bytes the context holds (workspace, staging, plans, spins)."""
    return load().lsg_memory_used(ctx)


LSG_NOALLOC_MAX_VERTICES = 1 << 20


def lsg_segment_noalloc(scan: lsg_scan, params: lsg_params, out: lsg_out, stream: int = 0) -> int:
    """lsg_segment with its workspace in the library's fixed device array, for
    callers that may not allocate device memory.  Returns the status code."""
    return load().lsg_segment_noalloc(ctypes.byref(scan), ctypes.byref(params), ctypes.byref(out),
                                      stream or None)


def lsg_noalloc_get_error(stream: int = 0) -> int:
    """Waits for the stream, reads and clears the device flags of the last
    lsg_segment_noalloc call on the current device; returns the status."""
    return load().lsg_noalloc_get_error(stream or None)


def lsg_spin_begin(ctx: int, scan: lsg_scan, params: lsg_params, out: lsg_out, stream: int = 0) -> int:
    h = _P()
    _check(load().lsg_spin_begin(ctx, ctypes.byref(scan), ctypes.byref(params), ctypes.byref(out),
                                 ctypes.byref(h), stream or None), "lsg_spin_begin")
    return h.value


def lsg_spin_push(spin: int, cols_ready: int, stream: int = 0) -> int:
    return load().lsg_spin_push(spin, cols_ready, stream or None)


def lsg_spin_finish(spin: int, stream: int = 0) -> int:
    return load().lsg_spin_finish(spin, stream or None)


def lsg_spin_destroy(spin: int) -> None:
    _check(load().lsg_spin_destroy(spin), "lsg_spin_destroy")


def lsg_raycast(spec: lsg_raycast_spec, xyzr: int, gt: int, stream: int = 0) -> int:
    """Ray-casts one synthetic scan into device buffers; returns the status."""
    return load().lsg_raycast(ctypes.byref(spec), xyzr, gt or None, stream or None)


# ---- convenience layer (torch for device memory and streams) -------------
@dataclass
class Params:
    """Python mirror of lsg_params with the library's defaults."""
    subsample: int = 1
    r_min: float = 0.0
    r_max: float = 100.0
    jump_rel_h: float = 0.10
    jump_rel_v: float = 1.0
    predicate: int = LSG_PRED_ANGLE
    angle_rad: float = math.radians(10.0)
    comp: Sequence[float] = (0.2, 0.2, 0.2)
    wrap: int = 1

    def to_c(self) -> lsg_params:
        p = lsg_params()
        p.subsample = int(self.subsample)
        p.r_min = float(self.r_min)
        p.r_max = float(self.r_max)
        p.jump_rel_h = float(self.jump_rel_h)
        p.jump_rel_v = float(self.jump_rel_v)
        p.predicate = int(self.predicate)
        p.angle_rad = float(self.angle_rad)
        for k in range(3):
            p.comp[k] = float(self.comp[k])
        p.wrap = int(self.wrap)
        return p


@dataclass
class Outputs:
    meshbits: "torch.Tensor"  # uint8 [H, Ws]
    normals: "torch.Tensor"   # float32 [H, Ws, 3]
    labels: "torch.Tensor"    # int32 [H, W]
    nseg: "torch.Tensor"      # int32 [1]

    def to_c(self) -> lsg_out:
        o = lsg_out()
        o.meshbits = self.meshbits.data_ptr() if self.meshbits.numel() else None
        o.normals = self.normals.data_ptr() if self.normals.numel() else None
        o.labels = self.labels.data_ptr() if self.labels.numel() else None
        o.nseg = self.nseg.data_ptr()
        return o


def ws_of(W: int, s: int) -> int:
    """Sampled columns ceil(W/s); 0 for an empty ring or an invalid s (which
    the library then rejects)."""
    return (W + s - 1) // s if (W > 0 and s >= 1) else 0


def alloc_outputs(H: int, W: int, s: int, device) -> Outputs:
    import torch
    Ws = ws_of(W, s)
    return Outputs(torch.empty((H, Ws), dtype=torch.uint8, device=device),
                   torch.empty((H, Ws, 3), dtype=torch.float32, device=device),
                   torch.empty((H, W), dtype=torch.int32, device=device),
                   torch.zeros(1, dtype=torch.int32, device=device))


def make_scan(elev, xyzr=None, range_=None, az0: float = 0.0, daz: float = 0.0) -> lsg_scan:
    """lsg_scan over device tensors (elev float32 [H]; xyzr float32 [H, W, 4]
    or range float32 [H, W])."""
    sc = lsg_scan()
    src = xyzr if xyzr is not None else range_
    sc.rings = int(src.shape[0])
    sc.cols = int(src.shape[1]) if src.dim() > 1 else 0
    sc.elevation = elev.data_ptr() if elev.numel() else None
    sc.azimuth0 = float(az0)
    sc.azimuth_step = float(daz)
    sc.xyzr = xyzr.data_ptr() if (xyzr is not None and xyzr.numel()) else None
    sc.range = range_.data_ptr() if (range_ is not None and range_.numel()) else None
    return sc


def _stream_ptr(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Context:
    """Owns an lsg context on one device."""

    def __init__(self, device: int = 0, budget_bytes: int = 0, tile: Optional[int] = None):
        self.device = device
        self.h = lsg_create(device, budget_bytes)
        if tile is not None:
            lsg_set_tile(self.h, tile)

    def close(self):
        if self.h:
            lsg_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def segment(self, elev, xyzr=None, range_=None, az0=0.0, daz=0.0, params: Params = Params(),
                out: Optional[Outputs] = None, stream=None) -> Outputs:
        src = xyzr if xyzr is not None else range_
        H, W = int(src.shape[0]), int(src.shape[1])
        if out is None:
            out = alloc_outputs(H, W, params.subsample, src.device)
        st = lsg_segment(self.h, make_scan(elev, xyzr, range_, az0, daz), params.to_c(), out.to_c(),
                         _stream_ptr(stream))
        _check(st, "lsg_segment")
        return out

    def label_from_mask(self, meshbits, valid, W: int, s: int, wrap: int, stream=None):
        import torch
        H = int(meshbits.shape[0])
        labels = torch.empty((H, W), dtype=torch.int32, device=meshbits.device)
        nseg = torch.zeros(1, dtype=torch.int32, device=meshbits.device)
        st = lsg_label_from_mask(self.h, H, W, s, wrap, meshbits.data_ptr() if meshbits.numel() else 0,
                                 valid.data_ptr() if (valid is not None and valid.numel()) else 0,
                                 labels.data_ptr() if labels.numel() else 0, nseg.data_ptr(),
                                 _stream_ptr(stream))
        _check(st, "lsg_label_from_mask")
        return labels, nseg

    def segment_stats(self, out: Outputs, W: int, s: int, min_points: int, normal_sums: bool = False, stream=None):
        """Sizes of out's segments (indexed by label), optional normal sums, and
        removal (in place) of segments of fewer than min_points points."""
        import torch
        H = int(out.labels.shape[0])
        dev = out.labels.device
        sizes = torch.empty(max(H * W, 1), dtype=torch.int32, device=dev)
        nsum = torch.empty((max(H * W, 1), 3), dtype=torch.float32, device=dev) if normal_sums else None
        nseg = torch.zeros(1, dtype=torch.int32, device=dev)
        st = load().lsg_segment_stats(self.h, H, W, s, min_points, out.labels.data_ptr() if out.labels.numel() else None,
                                      out.normals.data_ptr() if out.normals.numel() else None,
                                      out.meshbits.data_ptr() if out.meshbits.numel() else None, sizes.data_ptr(),
                                      nsum.data_ptr() if nsum is not None else None, nseg.data_ptr(),
                                      _stream_ptr(stream))
        _check(st, "lsg_segment_stats")
        return sizes, nsum, nseg

    def error(self) -> int:
        return lsg_get_error(self.h)

    def memory_used(self) -> int:
        return lsg_memory_used(self.h)


class Spin:
    """One revolution segmented while its columns arrive (lsg_spin_*): the
    caller fills the scan's input buffer column range by column range and
    calls push(cols_ready) after each, then finish(); the outputs equal
    Context.segment's."""

    def __init__(self, ctx: "Context", elev, xyzr=None, range_=None, az0=0.0, daz=0.0, params: "Params" = None,
                 out: Optional["Outputs"] = None, stream=None):
        params = params or Params()
        src = xyzr if xyzr is not None else range_
        H, W = int(src.shape[0]), int(src.shape[1])
        self.out = out if out is not None else alloc_outputs(H, W, params.subsample, src.device)
        self._keep = (make_scan(elev, xyzr, range_, az0, daz), params.to_c(), self.out.to_c())
        self.h = lsg_spin_begin(ctx.h, *self._keep, _stream_ptr(stream))

    def push(self, cols_ready: int, stream=None) -> None:
        _check(lsg_spin_push(self.h, cols_ready, _stream_ptr(stream)), "lsg_spin_push")

    def finish(self, stream=None) -> "Outputs":
        _check(lsg_spin_finish(self.h, _stream_ptr(stream)), "lsg_spin_finish")
        return self.out

    def close(self):
        if self.h:
            lsg_spin_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchPlan:
    """A captured batched pass over fixed device buffers; with ``io`` (one
    lsg_host_io per scan, pinned host buffers) and ``chunks``, the pass from
    and to host memory (lsg_batch_plan_io)."""

    def __init__(self, ctx: Context, scans: List[lsg_scan], params: List[lsg_params], outs: List[lsg_out],
                 tile: int = LSG_TILE_AUTO, io: Optional[List[lsg_host_io]] = None, chunks: int = 0):
        self.ctx = ctx
        self._keep = (scans, params, outs, io)
        if io is None:
            self.h = lsg_batch_plan(ctx.h, scans, params, outs, tile)
        else:
            self.h = lsg_batch_plan_io(ctx.h, scans, params, outs, io, chunks, tile)

    def io_bytes(self):
        """(host -> device, device -> host) bytes of one run of a host-buffer plan."""
        return lsg_plan_io_bytes(self.h)

    def run(self, stream=None):
        _check(lsg_batch_run(self.h, _stream_ptr(stream)), "lsg_batch_run")

    def autotune(self, reps: int = 3, stream=None):
        return lsg_autotune(self.h, reps, _stream_ptr(stream))

    @property
    def tile(self) -> int:
        return lsg_plan_tile(self.h)

    def set_fused(self, fused: bool):
        lsg_plan_set_fused(self.h, 1 if fused else 0)

    def set_schedule(self, schedule: int):
        """0 phased, 1 one persistent launch, 2 scan groups on overlapping branches."""
        lsg_plan_set_fused(self.h, int(schedule))

    @property
    def schedule(self) -> int:
        return load().lsg_plan_fused(self.h)

    @property
    def fused(self) -> bool:
        return load().lsg_plan_fused(self.h) == 1

    @property
    def launches(self) -> int:
        """Kernel launches in one run of the plan."""
        return load().lsg_plan_launches(self.h)

    def phase_times(self):
        """[ring order, tile kernel, border merge, labels] ms of the last replay."""
        return lsg_plan_phase_times(self.h)

    def close(self):
        if self.h:
            lsg_plan_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def raycast(elev, cols: int, az0: float, daz: float, prims, sigma: float, p_drop: float, r_max: float, seed: int,
            xyzr=None, gt=None, stream=None):
    """Synthetic scan on the device (lsg_raycast): elev a float32 device
    tensor [H] (radians), prims a float64 device tensor [n, 10]; returns
    (xyzr [H, W, 4] float32, gt [H, W] int32) device tensors."""
    import torch
    H = int(elev.shape[0])
    dev = elev.device
    if xyzr is None:
        xyzr = torch.empty((H, cols, 4), dtype=torch.float32, device=dev)
    if gt is None:
        gt = torch.empty((H, cols), dtype=torch.int32, device=dev)
    spec = lsg_raycast_spec()
    spec.rings, spec.cols = H, cols
    spec.elevation = elev.data_ptr() if H else None
    spec.azimuth0, spec.azimuth_step = az0, daz
    spec.nprims = int(prims.shape[0])
    spec.prims = prims.data_ptr() if spec.nprims else None
    spec.sigma, spec.p_drop, spec.r_max = sigma, p_drop, r_max
    spec.seed = seed & 0xFFFFFFFFFFFFFFFF
    _check(lsg_raycast(spec, xyzr.data_ptr(), gt.data_ptr(), _stream_ptr(stream)), "lsg_raycast")
    return xyzr, gt

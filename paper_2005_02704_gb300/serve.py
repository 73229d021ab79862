"""Serving path: continuous batching of scans from many sensors.

Scans arrive one by one (several sensors, each at its own rate).  The server
admits a scan as soon as a device slot for its shape is free or can be
allocated within the memory budget (admission by device memory), keeps slots
resident and reuses them for later scans of the same shape, and runs admitted
scans in batches on several CUDA streams ("lanes"): whenever a lane is idle
it takes every admitted scan waiting (up to ``max_batch``) and launches one
batched pass (``lsg_batch_launch``) for them, so scans that arrive while
others are on the GPU join the next batch and their work overlaps on the
device.  Each batch uploads its inputs, segments them, and copies labels and
segment counts back to pinned host memory on its lane's stream; a request is
complete when the host sees that stream's event.

The scheduler runs on the host; every step of the segmentation runs in the
library's kernels.  ``SlotPool`` holds the admission logic and is testable
without a GPU.
"""
from __future__ import annotations

import collections
import contextlib
import ctypes
import gc
import math
import time
from dataclasses import dataclass
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import lsg

ShapeKey = Tuple[int, int, int]  # rings, cols, subsample


def _block(nbytes: int) -> int:
    """Bytes the device allocator hands out for a tensor (512-byte blocks)."""
    return (max(int(nbytes), 1) + 511) // 512 * 512


def slot_bytes(key: ShapeKey) -> int:
    """Device bytes of one slot: its input and output tensors (x,y,z,r,
    elevations, mesh bytes, normals, labels, segment count).  The pass's
    workspace belongs to the lanes' contexts, which the server charges to the
    budget once, up front."""
    H, W, s = key
    Ws = lsg.ws_of(W, s)
    return (_block(H * W * 16) + _block(H * 4) + _block(H * Ws) + _block(H * Ws * 12) + _block(H * W * 4) +
            _block(4))


class SlotPool:
    """Resident device slots per scan shape under a byte budget.

    acquire(key) returns a free slot of that shape, allocating one when the
    budget allows (freeing idle slots of other shapes first if needed), or
    None when the request must wait.  release(slot) makes it free again.
    """

    def __init__(self, budget_bytes: int, alloc: Callable[[ShapeKey], object],
                 size_of: Callable[[ShapeKey], int] = slot_bytes, free_fn: Callable[[object], None] = None):
        self.budget = int(budget_bytes)
        self.alloc = alloc
        self.size_of = size_of
        self.free_fn = free_fn or (lambda s: None)
        self.free: Dict[ShapeKey, List[object]] = collections.defaultdict(list)
        self.used = 0
        self.live = 0        # slots handed out
        self.allocated = 0   # slots in existence
        self.peak = 0

    def acquire(self, key: ShapeKey):
        lst = self.free.get(key)
        if lst:
            self.live += 1
            return lst.pop()
        need = self.size_of(key)
        if need > self.budget:
            raise ValueError(f"a scan of shape {key} needs {need} bytes, more than the budget {self.budget}")
        if self.used + need > self.budget:
            # evict idle slots of other shapes, largest first
            idle = sorted(((self.size_of(k), k) for k, v in self.free.items() for _ in v), reverse=True)
            for sz, k in idle:
                if self.used + need <= self.budget:
                    break
                if k == key or not self.free[k]:
                    continue
                self.free_fn(self.free[k].pop())
                self.used -= sz
                self.allocated -= 1
        if self.used + need > self.budget:
            return None
        slot = self.alloc(key)
        self.used += need
        self.allocated += 1
        self.live += 1
        self.peak = max(self.peak, self.used)
        return slot

    def release(self, key: ShapeKey, slot) -> None:
        self.live -= 1
        self.free[key].append(slot)


@dataclass
class Request:
    ticket: int
    sensor: int
    key: ShapeKey
    host_xyzr: "torch.Tensor"      # pinned float32 [H, W, 4]
    host_elev: "torch.Tensor"      # pinned float32 [H]
    az0: float
    daz: float
    params: "lsg.Params"
    t_arrival: float               # wall clock (perf_counter)
    t_launch: float = 0.0
    t_done: float = 0.0
    slot: object = None
    keep_geometry: bool = False
    result: Optional[dict] = None
    c_params: object = None        # cached lsg_params of the sensor
    ref_params: object = None      # and a ctypes reference to it
    host_ptrs: object = None       # (x,y,z,r, elevations) host addresses


class Slot:
    """Device buffers of one request (inputs, outputs), pinned host buffers
    for its results, and the C descriptors pointing at them."""

    def __init__(self, key: ShapeKey, device):
        import torch
        H, W, s = key
        self.key = key
        self.xyzr = torch.empty((H, W, 4), dtype=torch.float32, device=device)
        self.elev = torch.empty(H, dtype=torch.float32, device=device)
        self.out = lsg.alloc_outputs(H, W, s, device)
        self.h_labels = torch.empty((H, W), dtype=torch.int32, pin_memory=True)
        self.h_nseg = torch.empty(1, dtype=torch.int32, pin_memory=True)
        self.h_meshbits = None
        self.h_normals = None
        self.c_out = self.out.to_c()
        self.c_scan = lsg.make_scan(self.elev, self.xyzr, None, 0.0, 0.0)
        self.c_io = lsg.lsg_host_io()
        self.c_io.labels = self.h_labels.data_ptr() if self.h_labels.numel() else None
        self.c_io.nseg = self.h_nseg.data_ptr()
        # references for the batch-of-one call, made once
        self.ref_scan, self.ref_out, self.ref_io = (ctypes.byref(self.c_scan), ctypes.byref(self.c_out),
                                                    ctypes.byref(self.c_io))

    def geometry_buffers(self):
        import torch
        if self.h_meshbits is None:
            self.h_meshbits = torch.empty(tuple(self.out.meshbits.shape), dtype=torch.uint8, pin_memory=True)
            self.h_normals = torch.empty(tuple(self.out.normals.shape), dtype=torch.float32, pin_memory=True)
        return self.h_meshbits, self.h_normals


class Server:
    """Continuous-batching server on one GPU."""

    def __init__(self, budget_bytes: int = 8 << 30, lanes: int = 3, max_batch: int = 64, device: int = 0,
                 max_shape: ShapeKey = (128, 4096, 1)):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.max_batch = max_batch
        # every lane's context, with workspace and staging sized for a full
        # batch of the largest expected scan (so that serving allocates
        # nothing but slots) and capped at the budget; what they hold is
        # charged to the budget first, and the slots share the rest
        H, W, s_ = max_shape
        Ws = lsg.ws_of(W, s_)
        tiles = ((H + 1) // 2 + 1) * (Ws // 120 + 1)  # the smallest tile shape: 2 x 120
        self.ctxs = [lsg.Context(device, budget_bytes=budget_bytes) for _ in range(lanes)]
        for c in self.ctxs:
            lsg.lsg_reserve(c.h, max_batch * lsg.scan_workspace_bytes(H, Ws), max_batch, 2 * max_batch * tiles)
        self.fixed_bytes = sum(c.memory_used() for c in self.ctxs)
        if self.fixed_bytes >= budget_bytes:
            raise ValueError(f"the lanes' workspace ({self.fixed_bytes} bytes) leaves nothing of the budget "
                             f"{budget_bytes} for scans")
        self.budget = int(budget_bytes)
        self.max_shape = max_shape
        self.shapes_ok = set()
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(lanes)]
        # what the batch-of-one launch passes, looked up once: the entry
        # point, the contexts' and streams' handles
        self._launch_io = lsg.load().lsg_batch_launch_io
        self._ctx_h = [c.h for c in self.ctxs]
        self._stream_h = [int(st.cuda_stream) for st in self.streams]
        self.events = [torch.cuda.Event() for _ in range(lanes)]
        self.inflight: List[Optional[List[Request]]] = [None] * lanes
        self.n_inflight = 0
        self.pool = SlotPool(budget_bytes - self.fixed_bytes, lambda k: Slot(k, self.device))
        # each lane's argument arrays, filled in place per batch
        self.c_args = [((lsg.lsg_scan * max_batch)(), (lsg.lsg_params * max_batch)(), (lsg.lsg_out * max_batch)(),
                        (lsg.lsg_host_io * max_batch)()) for _ in range(lanes)]
        self.pending: collections.deque = collections.deque()
        self.done: List[Request] = []
        self.batches = 0
        self.batch_sizes: List[int] = []

    def submit(self, req: Request) -> None:
        if req.key not in self.shapes_ok:
            H, W, s_ = req.key
            Hm, Wm, sm = self.max_shape
            if H * W > Hm * Wm or H * lsg.ws_of(W, s_) > Hm * lsg.ws_of(Wm, sm) or H > Hm:
                raise ValueError(f"scan shape {req.key} is larger than the server's largest shape {self.max_shape}")
            self.shapes_ok.add(req.key)
        self.pending.append(req)

    def busy(self) -> bool:
        return bool(self.pending) or self.n_inflight > 0

    def _reap(self) -> None:
        if not self.n_inflight:
            return
        for k, batch in enumerate(self.inflight):
            if batch is None or not self.events[k].query():
                continue
            now = time.perf_counter()
            for req in batch:
                req.t_done = now
                slot = req.slot
                if req.keep_geometry:
                    req.result = {"labels": slot.h_labels.clone(), "nseg": int(slot.h_nseg[0]),
                                  "meshbits": slot.h_meshbits.clone(), "normals": slot.h_normals.clone()}
                else:
                    req.result = {"nseg": int(slot.h_nseg[0])}
                self.pool.release(req.key, slot)
                req.slot = None
                self.done.append(req)
            self.inflight[k] = None
            self.n_inflight -= 1

    def _launch(self, k: int) -> bool:
        batch: List[Request] = []
        while self.pending and len(batch) < self.max_batch:
            req = self.pending[0]
            slot = self.pool.acquire(req.key)
            if slot is None:
                break  # admission waits for memory (first come, first served)
            self.pending.popleft()
            req.slot = slot
            batch.append(req)
        if not batch:
            return False
        st = self.streams[k]
        now = time.perf_counter()
        n = len(batch)
        if n == 1:
            # a batch of one passes the slot's own descriptors by reference
            # (references, handles and host addresses prepared beforehand: the
            # input copy is the call's first step, so every step before the
            # call delays the scan)
            req = batch[0]
            slot = req.slot
            req.t_launch = now
            sc = slot.c_scan
            sc.azimuth0 = req.az0
            sc.azimuth_step = req.daz
            h = slot.c_io
            if req.host_ptrs is not None:
                h.xyzr, h.elevation = req.host_ptrs
            else:
                h.xyzr = req.host_xyzr.data_ptr()
                h.elevation = req.host_elev.data_ptr()
            if req.keep_geometry:
                mbh, nrh = slot.geometry_buffers()
                h.meshbits = mbh.data_ptr() if mbh.numel() else None
                h.normals = nrh.data_ptr() if nrh.numel() else None
            else:
                h.meshbits = None
                h.normals = None
            prm = req.ref_params
            if prm is None:
                prm = ctypes.byref(req.c_params if req.c_params is not None else req.params.to_c())
            rc = self._launch_io(self._ctx_h[k], 1, slot.ref_scan, prm, slot.ref_out, slot.ref_io,
                                 self._stream_h[k])
            if rc != lsg.LSG_OK:
                raise lsg.LsgError(rc, "lsg_batch_launch_io")
            self.events[k].record(st)
            self.inflight[k] = batch
            self.n_inflight += 1
            self.batches += 1
            self.batch_sizes.append(1)
            return True
        scans, params, outs, io = self.c_args[k]
        for b, req in enumerate(batch):
            slot = req.slot
            req.t_launch = now
            sc = slot.c_scan
            sc.azimuth0 = req.az0
            sc.azimuth_step = req.daz
            scans[b] = sc
            params[b] = req.c_params if req.c_params is not None else req.params.to_c()
            outs[b] = slot.c_out
            h = slot.c_io
            h.xyzr = req.host_xyzr.data_ptr()
            h.elevation = req.host_elev.data_ptr()
            if req.keep_geometry:
                mbh, nrh = slot.geometry_buffers()
                h.meshbits = mbh.data_ptr() if mbh.numel() else None
                h.normals = nrh.data_ptr() if nrh.numel() else None
            else:
                h.meshbits = None
                h.normals = None
            io[b] = h
        # uploads, the batched pass and the result downloads, on this lane
        rc = lsg.load().lsg_batch_launch_io(self.ctxs[k].h, n, scans, params, outs, io, int(st.cuda_stream))
        if rc != lsg.LSG_OK:
            raise lsg.LsgError(rc, "lsg_batch_launch_io")
        self.events[k].record(st)
        self.inflight[k] = batch
        self.n_inflight += 1
        self.batches += 1
        self.batch_sizes.append(n)
        return True

    def poll(self) -> None:
        """Reap finished batches, then launch waiting scans on idle lanes."""
        self._reap()
        if self.pending:
            for k in range(len(self.inflight)):
                if self.inflight[k] is None and self.pending:
                    self._launch(k)

    def drain(self) -> None:
        while self.busy():
            self.poll()

    def close(self) -> None:
        self.torch.cuda.synchronize()
        for c in self.ctxs:
            c.close()


# --------------------------------------------------------------------------
# sensor simulation and the two serving loops
# --------------------------------------------------------------------------
@dataclass
class SensorFeed:
    """One simulated sensor: its scans (pinned host copies) and rate."""
    sensor: int
    key: ShapeKey
    rate_hz: float
    host_xyzr: List["torch.Tensor"]
    host_elev: "torch.Tensor"
    az0: float
    daz: float
    params: "lsg.Params"
    c_params: object = None
    ref_params: object = None
    host_ptrs: object = None       # (x,y,z,r, elevations) host address per scan


def arrival_trace(rates: Sequence[float], duration_s: float = 60.0, burst=(30.0, 40.0, 4.0),
                  seed: int = 7) -> List[Tuple[float, int]]:
    """Poisson arrivals (exponential gaps) per sensor, with the rate multiplied
    by burst[2] inside [burst[0], burst[1]).  Returns sorted (time, sensor)."""
    rng = np.random.default_rng(seed)
    out = []
    for k, r in enumerate(rates):
        t = float(rng.uniform(0.0, 1.0 / r))
        while t < duration_s:
            out.append((t, k))
            rate = r * (burst[2] if burst and burst[0] <= t < burst[1] else 1.0)
            t += float(rng.exponential(1.0 / rate))
    out.sort()
    return out


def _request(feed: SensorFeed, ticket: int, t_arrival: float, keep_geometry: bool = False) -> Request:
    m = ticket % len(feed.host_xyzr)
    if feed.c_params is None:
        feed.c_params = feed.params.to_c()
        feed.ref_params = ctypes.byref(feed.c_params)
        e = feed.host_elev.data_ptr()
        feed.host_ptrs = [(x.data_ptr(), e) for x in feed.host_xyzr]
    return Request(ticket, feed.sensor, feed.key, feed.host_xyzr[m], feed.host_elev, feed.az0, feed.daz,
                   feed.params, t_arrival, keep_geometry=keep_geometry, c_params=feed.c_params,
                   ref_params=feed.ref_params, host_ptrs=feed.host_ptrs[m])


@contextlib.contextmanager
def no_gc_pauses():
    """Pauses Python's cyclic garbage collector (after moving the objects that
    exist now out of its reach) for a latency-sensitive host loop: a full
    collection over a large heap stalls the loop for milliseconds.  The loop
    creates no reference cycles, so nothing is left for the collector."""
    was = gc.isenabled()
    gc.collect()
    gc.freeze()
    gc.disable()
    try:
        yield
    finally:
        if was:
            gc.enable()
        gc.unfreeze()


def run_served(server: Server, feeds: Sequence[SensorFeed], trace, time_scale: float,
               keep_geometry: bool = False) -> dict:
    """Replays the trace (virtual seconds / time_scale = wall seconds) through
    the server; returns latency and throughput statistics."""
    with no_gc_pauses():
        return _run_served(server, feeds, trace, time_scale, keep_geometry)


def _run_served(server: Server, feeds: Sequence[SensorFeed], trace, time_scale: float,
                keep_geometry: bool) -> dict:
    clock = time.perf_counter
    t0 = clock()
    i, n = 0, len(trace)
    reqs = []
    while i < n or server.pending or server.n_inflight:
        now = clock()
        while i < n and trace[i][0] / time_scale <= now - t0:
            tv, k = trace[i]
            r = _request(feeds[k], i, t0 + tv / time_scale, keep_geometry)
            reqs.append(r)
            server.submit(r)
            i += 1
        server.poll()
    t1 = time.perf_counter()
    return summarize(reqs, t1 - t0)


def run_serial(feeds: Sequence[SensorFeed], trace, time_scale: float, device: int = 0) -> dict:
    """The plain per-scan loop: one scan at a time in arrival order (upload,
    lsg_segment, download, synchronise), on one stream."""
    with no_gc_pauses():
        return _run_serial(feeds, trace, time_scale, device)


def _run_serial(feeds: Sequence[SensorFeed], trace, time_scale: float, device: int) -> dict:
    import torch
    dev = torch.device("cuda", device)
    ctx = lsg.Context(device)
    slots: Dict[ShapeKey, Slot] = {}
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    reqs = []
    for i, (tv, k) in enumerate(trace):
        arrival = t0 + tv / time_scale
        while time.perf_counter() < arrival:
            pass
        feed = feeds[k]
        r = _request(feed, i, arrival)
        slot = slots.get(feed.key)
        if slot is None:
            slot = slots[feed.key] = Slot(feed.key, dev)
        r.t_launch = time.perf_counter()
        slot.xyzr.copy_(r.host_xyzr, non_blocking=True)
        slot.elev.copy_(r.host_elev, non_blocking=True)
        ctx.segment(slot.elev, xyzr=slot.xyzr, az0=r.az0, daz=r.daz, params=r.params, out=slot.out,
                    stream=stream)
        slot.h_labels.copy_(slot.out.labels, non_blocking=True)
        slot.h_nseg.copy_(slot.out.nseg, non_blocking=True)
        stream.synchronize()
        r.t_done = time.perf_counter()
        reqs.append(r)
    t1 = time.perf_counter()
    ctx.close()
    return summarize(reqs, t1 - t0)


def device_footprint(server: Server) -> int:
    """Device bytes the server holds now: its lanes' contexts and its slots."""
    return sum(c.memory_used() for c in server.ctxs) + server.pool.used


def summarize(reqs: Sequence[Request], wall_s: float) -> dict:
    lat = np.array([(r.t_done - r.t_arrival) * 1e3 for r in reqs]) if reqs else np.zeros(1)
    pts = sum(r.key[0] * r.key[1] for r in reqs)
    by_shape: Dict[str, List[float]] = {}
    for r, x in zip(reqs, lat):
        by_shape.setdefault(f"{r.key[0]}x{r.key[1]}" + (f"_s{r.key[2]}" if r.key[2] != 1 else ""), []).append(x)
    return {"scans": len(reqs), "points": pts, "wall_s": wall_s, "scans_per_s": len(reqs) / wall_s,
            "points_per_s": pts / wall_s, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()),
            "p50_ms_by_shape": {k: float(np.percentile(v, 50)) for k, v in sorted(by_shape.items())}}


def make_feeds(specs, scans_per_sensor: int = 4, seed: int = 11) -> List[SensorFeed]:
    """Sensors from lidarsim specs: each gets `scans_per_sensor` ray-cast scans
    (pinned host memory) and a rate drawn from 10-20 Hz."""
    import torch
    import lidarsim
    from dataclasses import replace
    rng = np.random.default_rng(seed)
    feeds = []
    for k, sp in enumerate(specs):
        xs = []
        scan = None
        for m in range(scans_per_sensor):
            scan = lidarsim.make_scan(replace(sp, seed=sp.seed * 1000 + m))
            t = torch.empty(scan.xyzr.shape, dtype=torch.float32, pin_memory=True)
            t.numpy()[:] = scan.xyzr
            xs.append(t)
        e = torch.empty(scan.elev.shape, dtype=torch.float32, pin_memory=True)
        e.numpy()[:] = scan.elev
        p = lsg.Params(subsample=sp.subsample, r_max=sp.r_max, jump_rel_h=sp.jump_rel_h, jump_rel_v=sp.jump_rel_v,
                       angle_rad=math.radians(sp.angle_deg))
        feeds.append(SensorFeed(k, (scan.rings, scan.cols, sp.subsample), float(rng.uniform(10.0, 20.0)), xs, e,
                                scan.az0, scan.daz, p))
    return feeds

"""Packed device buffers for a batch of scans (plumbing for the batched and
served paths).

All scans' inputs live in one device buffer (x,y,z,r float32, 16-byte
aligned per scan, or, for range-only decoding, the ranges alone) plus one
buffer of elevations; all outputs in one buffer per kind.  ``lsg_scan`` / ``lsg_out`` descriptors point into them, so one
``lsg_batch_plan`` covers the whole batch and replays stay valid as long as
the buffers live.  A pinned host mirror of the inputs and of the labels and
segment counts serves the end-to-end (host -> device -> host) path, which
``HostPipeline`` runs in chunks so that copies in both directions overlap the
passes.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Sequence

import numpy as np

from . import lsg


@dataclass
class ScanShape:
    rings: int
    cols: int
    subsample: int

    @property
    def ws(self) -> int:
        return lsg.ws_of(self.cols, self.subsample)

    @property
    def points(self) -> int:
        return self.rings * self.cols

    @property
    def vertices(self) -> int:
        return self.rings * self.ws


class DeviceBatch:
    """form "xyzr": x,y,z,r float32 per point; "range": the range alone (the
    library computes x,y,z from the ring elevation and the column azimuth)."""

    def __init__(self, shapes: Sequence[ScanShape], params: Sequence["lsg.Params"], device=0,
                 pinned: bool = True, form: str = "xyzr"):
        import torch
        if form not in ("xyzr", "range"):
            raise ValueError(f"unknown input form {form!r}")
        self.form = form
        self.in_width = 4 if form == "xyzr" else 1  # float32 values per input point
        self.torch = torch
        self.dev = torch.device("cuda", device) if isinstance(device, int) else device
        self.n = len(shapes)
        self.shapes = list(shapes)
        self.params = list(params)
        self.pt_off = np.zeros(self.n + 1, np.int64)
        self.v_off = np.zeros(self.n + 1, np.int64)
        self.e_off = np.zeros(self.n + 1, np.int64)
        for b, sh in enumerate(self.shapes):
            self.pt_off[b + 1] = self.pt_off[b] + sh.points
            self.v_off[b + 1] = self.v_off[b] + sh.vertices
            self.e_off[b + 1] = self.e_off[b] + sh.rings
        P, V, E = int(self.pt_off[-1]), int(self.v_off[-1]), int(self.e_off[-1])
        self.points = P
        self.vertices = V
        f32, i32, u8 = torch.float32, torch.int32, torch.uint8
        self.d_in = torch.empty((max(P, 1), self.in_width), dtype=f32, device=self.dev)
        self.d_elev = torch.empty(max(E, 1), dtype=f32, device=self.dev)
        self.d_mb = torch.empty(max(V, 1), dtype=u8, device=self.dev)
        self.d_nrm = torch.empty((max(V, 1), 3), dtype=f32, device=self.dev)
        self.d_lab = torch.empty(max(P, 1), dtype=i32, device=self.dev)
        self.d_nseg = torch.zeros(max(self.n, 1), dtype=i32, device=self.dev)
        self.h_in = torch.empty((max(P, 1), self.in_width), dtype=f32, pin_memory=pinned)
        self.h_elev = torch.empty(max(E, 1), dtype=f32, pin_memory=pinned)
        self.h_lab = torch.empty(max(P, 1), dtype=i32, pin_memory=pinned)
        self.h_nseg = torch.empty(max(self.n, 1), dtype=i32, pin_memory=pinned)
        self.az0 = np.zeros(self.n, np.float32)
        self.daz = np.zeros(self.n, np.float32)

    # ---- host staging -----------------------------------------------------
    def set_scan(self, b: int, scan) -> None:
        """Copy a lidarsim.Scan into slot b of the pinned host mirror."""
        sh = self.shapes[b]
        assert scan.rings == sh.rings and scan.cols == sh.cols
        p0, p1 = self.pt_off[b], self.pt_off[b + 1]
        src = scan.xyzr if self.form == "xyzr" else scan.range
        self.h_in[p0:p1].numpy()[:] = src.reshape(-1, self.in_width)
        e0, e1 = self.e_off[b], self.e_off[b + 1]
        self.h_elev[e0:e1].numpy()[:] = scan.elev
        self.az0[b] = scan.az0
        self.daz[b] = scan.daz

    def upload(self, stream=None, non_blocking: bool = True) -> int:
        """Host -> device copy of every input; returns the bytes copied."""
        torch = self.torch
        with torch.cuda.stream(stream) if stream is not None else _null():
            self.d_in.copy_(self.h_in, non_blocking=non_blocking)
            self.d_elev.copy_(self.h_elev, non_blocking=non_blocking)
        return self.h_in.numel() * 4 + self.h_elev.numel() * 4

    def download(self, stream=None, non_blocking: bool = True) -> int:
        """Device -> host copy of the labels and segment counts; returns bytes."""
        torch = self.torch
        with torch.cuda.stream(stream) if stream is not None else _null():
            self.h_lab.copy_(self.d_lab, non_blocking=non_blocking)
            self.h_nseg.copy_(self.d_nseg, non_blocking=non_blocking)
        return self.h_lab.numel() * 4 + self.h_nseg.numel() * 4

    # ---- descriptors ------------------------------------------------------
    def c_scans(self) -> List["lsg.lsg_scan"]:
        out = []
        for b, sh in enumerate(self.shapes):
            sc = lsg.lsg_scan()
            sc.rings, sc.cols = sh.rings, sh.cols
            sc.elevation = self.d_elev.data_ptr() + 4 * int(self.e_off[b]) if sh.rings else None
            sc.azimuth0 = float(self.az0[b])
            sc.azimuth_step = float(self.daz[b])
            ptr = self.d_in.data_ptr() + 4 * self.in_width * int(self.pt_off[b]) if sh.points else None
            sc.xyzr = ptr if self.form == "xyzr" else None
            sc.range = ptr if self.form == "range" else None
            out.append(sc)
        return out

    def c_outs(self) -> List["lsg.lsg_out"]:
        out = []
        for b, sh in enumerate(self.shapes):
            o = lsg.lsg_out()
            v0 = int(self.v_off[b])
            p0 = int(self.pt_off[b])
            o.meshbits = self.d_mb.data_ptr() + v0 if sh.vertices else None
            o.normals = self.d_nrm.data_ptr() + 12 * v0 if sh.vertices else None
            o.labels = self.d_lab.data_ptr() + 4 * p0 if sh.points else None
            o.nseg = self.d_nseg.data_ptr() + 4 * b
            out.append(o)
        return out

    def c_params(self) -> List["lsg.lsg_params"]:
        return [p.to_c() for p in self.params]

    def plan(self, ctx: "lsg.Context", tile: int = lsg.LSG_TILE_AUTO) -> "lsg.BatchPlan":
        return lsg.BatchPlan(ctx, self.c_scans(), self.c_params(), self.c_outs(), tile)

    def pipeline(self, ctx: "lsg.Context", tile: int = lsg.LSG_TILE_AUTO, chunks: int = 8,
                 schedule=None) -> "HostPipeline":
        return HostPipeline(self, ctx, tile, chunks, schedule)

    # ---- per-scan views of the device outputs -----------------------------
    def view(self, b: int):
        sh = self.shapes[b]
        v0, v1 = int(self.v_off[b]), int(self.v_off[b + 1])
        p0, p1 = int(self.pt_off[b]), int(self.pt_off[b + 1])
        return (self.d_mb[v0:v1].view(sh.rings, sh.ws), self.d_nrm[v0:v1].view(sh.rings, sh.ws, 3),
                self.d_lab[p0:p1].view(sh.rings, sh.cols), self.d_nseg[b:b + 1])

    def scan_inputs(self, b: int):
        sh = self.shapes[b]
        p0, p1 = int(self.pt_off[b]), int(self.pt_off[b + 1])
        e0, e1 = int(self.e_off[b]), int(self.e_off[b + 1])
        if self.form == "range":
            return self.d_elev[e0:e1], self.d_in[p0:p1].view(sh.rings, sh.cols)
        return self.d_elev[e0:e1], self.d_in[p0:p1].view(sh.rings, sh.cols, 4)


class HostPipeline:
    """End-to-end passes from the pinned host mirror, in chunks that overlap.

    The batch is cut into ``chunks`` runs of consecutive scans with about
    equal point counts, each with its own captured plan.  In a step, chunk c's
    inputs go host -> device on one stream, its pass runs on a second stream
    once they have landed, and its labels and segment counts go device ->
    host on a third once the pass is done, so the copies of the neighbouring
    chunks, in both directions, run under each chunk's pass.  A step starts
    after the work already queued on the caller's stream and the caller's
    stream waits for its last copy.
    """

    def __init__(self, db: DeviceBatch, ctx: "lsg.Context", tile: int = lsg.LSG_TILE_AUTO, chunks: int = 8,
                 schedule=None):
        torch = db.torch
        self.db = db
        n = db.n
        chunks = max(1, min(int(chunks), n))
        bounds = [0]
        for c in range(1, chunks):
            b = int(np.searchsorted(db.pt_off, db.points * c / chunks))
            b = max(bounds[-1] + 1, min(b, n - (chunks - c)))
            bounds.append(b)
        bounds.append(n)
        self.ranges = [(b0, b1) for b0, b1 in zip(bounds[:-1], bounds[1:]) if b1 > b0]
        scans, params, outs = db.c_scans(), db.c_params(), db.c_outs()
        self.plans = [lsg.BatchPlan(ctx, scans[b0:b1], params[b0:b1], outs[b0:b1], tile) for b0, b1 in self.ranges]
        if schedule is not None:
            for p in self.plans:
                p.set_schedule(int(schedule))
        self.s_in = torch.cuda.Stream(db.dev)
        self.s_run = torch.cuda.Stream(db.dev)
        self.s_out = torch.cuda.Stream(db.dev)
        self.ev_in = [torch.cuda.Event() for _ in self.ranges]
        self.ev_run = [torch.cuda.Event() for _ in self.ranges]
        self.ev_out = torch.cuda.Event()

    def step(self, stream=None):
        """One end-to-end pass; returns (host->device bytes, device->host bytes)."""
        torch, db = self.db.torch, self.db
        cur = stream if stream is not None else torch.cuda.current_stream(db.dev)
        self.s_in.wait_stream(cur)
        self.s_run.wait_stream(cur)
        self.s_out.wait_stream(cur)
        with torch.cuda.stream(self.s_in):
            db.d_elev.copy_(db.h_elev, non_blocking=True)
        h2d, d2h = db.h_elev.numel() * 4, 0
        for c, (b0, b1) in enumerate(self.ranges):
            p0, p1 = int(db.pt_off[b0]), int(db.pt_off[b1])
            with torch.cuda.stream(self.s_in):
                db.d_in[p0:p1].copy_(db.h_in[p0:p1], non_blocking=True)
                self.ev_in[c].record(self.s_in)
            self.s_run.wait_event(self.ev_in[c])
            self.plans[c].run(stream=self.s_run)
            self.ev_run[c].record(self.s_run)
            self.s_out.wait_event(self.ev_run[c])
            with torch.cuda.stream(self.s_out):
                db.h_lab[p0:p1].copy_(db.d_lab[p0:p1], non_blocking=True)
                db.h_nseg[b0:b1].copy_(db.d_nseg[b0:b1], non_blocking=True)
            h2d += (p1 - p0) * 4 * db.in_width
            d2h += (p1 - p0) * 4 + (b1 - b0) * 4
        self.ev_out.record(self.s_out)
        cur.wait_event(self.ev_out)
        return h2d, d2h

    def close(self) -> None:
        for p in self.plans:
            p.close()
        self.plans = []


class _null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False

"""Packed device buffers for a batch of scans (plumbing for the batched and
served paths).

All scans' inputs live in one device buffer (x,y,z,r float32, 16-byte
aligned per scan, or, for range-only decoding, the ranges alone) plus one
buffer of elevations; all outputs in one buffer per kind.  ``lsg_scan`` / ``lsg_out`` descriptors point into them, so one
``lsg_batch_plan`` covers the whole batch and replays stay valid as long as
the buffers live.  A pinned host mirror of the inputs and of every output
(labels, segment counts, mesh bytes, normals) serves the end-to-end path,
``lsg_batch_plan_io``: one captured graph per step that copies the inputs in,
runs the pass and copies every output back, in chunks whose copies in both
directions overlap the other chunks' passes.
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
        self.h_mb = torch.empty(max(V, 1), dtype=u8, pin_memory=pinned)
        self.h_nrm = torch.empty((max(V, 1), 3), dtype=f32, pin_memory=pinned)
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

    def c_host_io(self) -> List["lsg.lsg_host_io"]:
        """Host buffers of every scan in the pinned mirrors (inputs in the
        batch's form, every output)."""
        out = []
        for b, sh in enumerate(self.shapes):
            io = lsg.lsg_host_io()
            p0, v0, e0 = int(self.pt_off[b]), int(self.v_off[b]), int(self.e_off[b])
            io.xyzr = self.h_in.data_ptr() + 4 * self.in_width * p0 if sh.points else None
            io.elevation = self.h_elev.data_ptr() + 4 * e0 if sh.rings else None
            io.labels = self.h_lab.data_ptr() + 4 * p0 if sh.points else None
            io.nseg = self.h_nseg.data_ptr() + 4 * b
            io.meshbits = self.h_mb.data_ptr() + v0 if sh.vertices else None
            io.normals = self.h_nrm.data_ptr() + 12 * v0 if sh.vertices else None
            out.append(io)
        return out

    def plan_io(self, ctx: "lsg.Context", tile: int = lsg.LSG_TILE_AUTO, chunks: int = 16) -> "lsg.BatchPlan":
        """The end-to-end plan: host inputs in, every output back to the
        pinned host mirrors, in one graph replay per step."""
        return lsg.BatchPlan(ctx, self.c_scans(), self.c_params(), self.c_outs(), tile, io=self.c_host_io(),
                             chunks=chunks)

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


class _null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False

"""GPU tests of the batched path: one captured pass over many uneven scans
equals the per-scan path bit for bit, the autotuner keeps results, and the
benchmark workload (512 scans) matches the oracle on sampled scans and on
every scan's labels given its own mask."""
import math

import numpy as np
import pytest

import lidarsim
import oracle as O
import parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def mods():
    from paper_2005_02704_gb300 import batch, lsg
    return lsg, batch


def params_of(spec):
    lsg, _ = mods()
    return lsg.Params(subsample=spec.subsample, r_max=spec.r_max, jump_rel_h=spec.jump_rel_h,
                      jump_rel_v=spec.jump_rel_v, angle_rad=math.radians(spec.angle_deg))


def make_batch(specs, scans, form="xyzr"):
    lsg, batch = mods()
    shapes = [batch.ScanShape(s.rings, s.cols, sp.subsample) for sp, s in zip(specs, scans)]
    db = batch.DeviceBatch(shapes, [params_of(sp) for sp in specs], 0, form=form)
    for b, s in enumerate(scans):
        db.set_scan(b, s)
    db.upload()
    torch.cuda.synchronize()
    return db


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    lsg, _ = mods()
    c = lsg.Context(0)
    yield c
    c.close()


def mixed_specs(n, seed0):
    specs = lidarsim.batch_specs(n, seed0)
    # add sub-sampling, no-wrap-sized and tiny scans to the mix
    from dataclasses import replace
    specs[1] = replace(specs[1], subsample=3)
    specs[2] = replace(specs[2], elev_deg=specs[2].elev_deg[:1], cols=5)
    specs[3] = replace(specs[3], cols=2)
    return specs


@pytest.mark.parametrize("schedule", [1, 0, 2], ids=["fused", "phased", "grouped"])
@pytest.mark.parametrize("tile", ["16x240", "32x120", "32x240", "32x480", "64x240", "16x120", "8x120", "4x120",
                                  "2x120"])
def test_batch_equals_per_scan(ctx, tile, schedule):
    lsg, _ = mods()
    specs = mixed_specs(12, 5000)
    scans = [lidarsim.make_scan(sp) for sp in specs]
    db = make_batch(specs, scans)
    plan = db.plan(ctx, lsg.TILES[tile])
    plan.set_schedule(schedule)
    assert plan.schedule == schedule
    plan.run()
    plan.run()  # replays are idempotent
    torch.cuda.synchronize()
    assert ctx.error() == lsg.LSG_OK
    for b, (sp, s) in enumerate(zip(specs, scans)):
        mb, nrm, lab, nseg = db.view(b)
        elev, xyzr = db.scan_inputs(b)
        out = ctx.segment(elev, xyzr=xyzr, az0=s.az0, daz=s.daz, params=params_of(sp))
        torch.cuda.synchronize()
        assert torch.equal(out.meshbits, mb)
        assert torch.equal(out.normals, nrm)
        assert torch.equal(out.labels, lab)
        assert torch.equal(out.nseg, nseg)
    plan.close()


@pytest.mark.parametrize("schedule", [1, 0, 2], ids=["fused", "phased", "grouped"])
def test_range_input_batch_equals_per_scan(ctx, schedule):
    """Range-only decoding in a batch (x,y,z from the ring elevation and the
    column azimuth) equals the per-scan range-only path bit for bit, and the
    host-buffer plan (lsg_batch_plan_io) over range inputs gives the same
    outputs in host memory."""
    lsg, _ = mods()
    specs = mixed_specs(10, 5600)
    scans = [lidarsim.make_scan(sp) for sp in specs]
    db = make_batch(specs, scans, form="range")
    plan = db.plan(ctx)
    plan.set_schedule(schedule)
    plan.run()
    torch.cuda.synchronize()
    assert ctx.error() == lsg.LSG_OK
    for b, (sp, s) in enumerate(zip(specs, scans)):
        mb, nrm, lab, nseg = db.view(b)
        elev, rng = db.scan_inputs(b)
        assert rng.shape == (s.rings, s.cols)
        out = ctx.segment(elev, range_=rng, az0=s.az0, daz=s.daz, params=params_of(sp))
        torch.cuda.synchronize()
        assert torch.equal(out.meshbits, mb) and torch.equal(out.normals, nrm)
        assert torch.equal(out.labels, lab) and torch.equal(out.nseg, nseg)
    want = [t.cpu().clone() for t in (db.d_lab, db.d_nseg, db.d_mb, db.d_nrm)]
    db.d_lab.fill_(-7)
    pio = db.plan_io(ctx, chunks=3)
    pio.run()
    torch.cuda.synchronize()
    assert ctx.error() == lsg.LSG_OK
    h2d, d2h = pio.io_bytes()
    assert h2d == db.points * 4 + db.h_elev.numel() * 4
    assert d2h == db.points * 4 + db.n * 4 + db.vertices * 13
    for got, w in zip((db.h_lab, db.h_nseg, db.h_mb, db.h_nrm), want):
        assert torch.equal(got, w)
    pio.close()
    plan.close()


def test_autotune_keeps_results(ctx):
    lsg, _ = mods()
    specs = mixed_specs(8, 6000)
    scans = [lidarsim.make_scan(sp) for sp in specs]
    db = make_batch(specs, scans)
    plan = db.plan(ctx)
    plan.run()
    torch.cuda.synchronize()
    ref = (db.d_mb.clone(), db.d_nrm.clone(), db.d_lab.clone(), db.d_nseg.clone())
    best, ms = plan.autotune(reps=2)
    assert 0 <= best < lsg.LSG_TILE_COUNT and plan.tile == best and ms > 0
    plan.run()
    torch.cuda.synchronize()
    for a, b in zip(ref, (db.d_mb, db.d_nrm, db.d_lab, db.d_nseg)):
        assert torch.equal(a, b)
    plan.close()


def test_bench_workload_512_scans(ctx):
    """The benchmark's batch (512 seeded scans, rings 16..128, widths
    1024..4096) in the benchmark's launch configuration: sampled scans
    against the full oracle; every scan's labels and segment count against
    the oracle's components of the GPU's own mask."""
    lsg, _ = mods()
    specs = lidarsim.batch_specs(512)
    scans = [lidarsim.make_scan(sp) for sp in specs]
    db = make_batch(specs, scans)
    plan = db.plan(ctx, lsg.TILES["32x120"])
    plan.set_schedule(2)  # the autotuner's choice for this batch: grouped, 32 x 120 tiles
    assert plan.tile == lsg.TILES["32x120"] and plan.schedule == 2
    plan.run()
    torch.cuda.synchronize()
    assert ctx.error() == lsg.LSG_OK
    mb_all = db.d_mb.cpu().numpy()
    nrm_all = db.d_nrm.cpu().numpy()
    lab_all = db.d_lab.cpu().numpy()
    nseg_all = db.d_nseg.cpu().numpy()
    for b, (sp, s) in enumerate(zip(specs, scans)):
        H, W, Ws = s.rings, s.cols, lsg.ws_of(s.cols, sp.subsample)
        v0, p0 = int(db.v_off[b]), int(db.pt_off[b])
        mb = mb_all[v0:v0 + H * Ws].reshape(H, Ws)
        lab = lab_all[p0:p0 + H * W].reshape(H, W)
        order = O.ring_order(s.elev)
        valid = parity.sorted_valid(s, params_of(sp), order)
        want, n = O.label_from_mask(mb, valid, W, sp.subsample, 1)
        assert np.array_equal(lab, want), b
        assert nseg_all[b] == n
        if b % 64 == 0:  # sampled full comparison
            p = params_of(sp)
            orc = O.segment_scan(s, parity.oracle_params(p))
            bounds = parity.normal_bounds(orc)
            nrm = nrm_all[v0:v0 + H * Ws].reshape(H, Ws, 3)
            parity.compare_geometry(mb, nrm, orc, parity.oracle_params(p), bounds)
    plan.close()


@pytest.mark.parametrize("chunks", [1, 3, 8, 64])
def test_host_buffer_plan_equals_plan(ctx, chunks):
    """The end-to-end plan (lsg_batch_plan_io: host inputs copied in, the pass,
    every output copied back, in chunks) leaves the device plan's labels,
    segment counts, mesh bytes and normals in the pinned host buffers, and
    declares the bytes it moves.  Each of two replays starts from zeroed
    device inputs and host outputs, so each must copy in both directions."""
    lsg, _ = mods()
    specs = mixed_specs(10, 7000)
    scans = [lidarsim.make_scan(sp) for sp in specs]
    db = make_batch(specs, scans)
    plan = db.plan(ctx, lsg.TILES["32x120"])
    plan.set_fused(False)
    plan.run()
    torch.cuda.synchronize()
    want = [t.cpu().clone() for t in (db.d_lab, db.d_nseg, db.d_mb, db.d_nrm)]
    for t in (db.d_lab, db.d_nseg, db.d_mb, db.d_nrm, db.d_in):
        t.fill_(0)
    pio = db.plan_io(ctx, lsg.TILES["32x120"], chunks=chunks)
    assert pio.launches == 4 * min(chunks, db.n)
    h2d, d2h = pio.io_bytes()
    assert h2d == db.points * 16 + db.h_elev.numel() * 4
    assert d2h == db.points * 4 + db.n * 4 + db.vertices * 13
    for rep in range(2):
        db.d_in.fill_(0)
        torch.cuda.synchronize()
        for t in (db.h_lab, db.h_nseg, db.h_mb, db.h_nrm):
            t.fill_(0)
        pio.run()
        torch.cuda.synchronize()
        assert ctx.error() == lsg.LSG_OK
        for got, w in zip((db.h_lab, db.h_nseg, db.h_mb, db.h_nrm), want):
            assert torch.equal(got, w), rep
    pio.close()
    plan.close()


def test_host_buffer_plan_rejects_pageable_memory(ctx):
    lsg, batch = mods()
    specs = lidarsim.batch_specs(2, 7100)
    scans = [lidarsim.make_scan(sp) for sp in specs]
    shapes = [batch.ScanShape(s.rings, s.cols, sp.subsample) for sp, s in zip(specs, scans)]
    db = batch.DeviceBatch(shapes, [params_of(sp) for sp in specs], 0, pinned=False)
    with pytest.raises(lsg.LsgError) as ei:
        db.plan_io(ctx, chunks=2)
    assert ei.value.status == lsg.LSG_E_ARG


@pytest.mark.parametrize("schedule", [1, 0, 2], ids=["fused", "phased", "grouped"])
def test_batch_with_empty_scans(ctx, schedule):
    """Scans without points (no rings, or no columns) inside a batch get zero
    segments and leave their neighbours' results unchanged."""
    lsg, batch = mods()
    specs = mixed_specs(6, 7300)
    scans = [lidarsim.make_scan(sp) for sp in specs]
    shapes = [batch.ScanShape(s.rings, s.cols, sp.subsample) for sp, s in zip(specs, scans)]
    # an empty scan first, in the middle and last
    shapes = [batch.ScanShape(0, 64, 1)] + shapes[:3] + [batch.ScanShape(8, 0, 1)] + shapes[3:] + \
        [batch.ScanShape(0, 0, 1)]
    order = [None, 0, 1, 2, None, 3, 4, 5, None]
    params = [params_of(specs[k]) if k is not None else lsg.Params() for k in order]
    db = batch.DeviceBatch(shapes, params, 0)
    for b, k in enumerate(order):
        if k is not None:
            db.set_scan(b, scans[k])
    db.upload()
    db.d_nseg.fill_(-1)
    torch.cuda.synchronize()
    plan = db.plan(ctx, lsg.TILES["32x120"])
    plan.set_schedule(schedule)
    # kernel launches per run: phased 4, fused 1, grouped ring order + 3 per scan group
    if schedule == 2:
        assert plan.launches in (4, 7, 10, 13)
    else:
        assert plan.launches == (1 if schedule == 1 else 4)
    plan.run()
    torch.cuda.synchronize()
    assert ctx.error() == lsg.LSG_OK
    for b, k in enumerate(order):
        mb, nrm, lab, nseg = db.view(b)
        if k is None:
            assert int(nseg.item()) == 0
            continue
        elev, xyzr = db.scan_inputs(b)
        out = ctx.segment(elev, xyzr=xyzr, az0=scans[k].az0, daz=scans[k].daz, params=params_of(specs[k]))
        torch.cuda.synchronize()
        assert torch.equal(out.labels, lab) and torch.equal(out.nseg, nseg) and torch.equal(out.meshbits, mb)
    plan.close()

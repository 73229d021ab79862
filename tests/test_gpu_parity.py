"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bars (derived in tests/parity.py): mesh connectivity bit-exact; normals within
1e-4 rad on well-conditioned vertices and within their derived FP32 bound on
the rest; edge predicates equal outside the stated margin band; labels
bit-exact given the same edge mask, both ways.
"""
import math
from dataclasses import replace

import numpy as np
import pytest

import lidarsim
import oracle as O
import parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def lsg_mod():
    from paper_2005_02704_gb300 import lsg
    return lsg


def params_of(spec, **kw):
    lsg = lsg_mod()
    p = lsg.Params(subsample=spec.subsample, r_max=spec.r_max, jump_rel_h=spec.jump_rel_h,
                   jump_rel_v=spec.jump_rel_v, angle_rad=math.radians(spec.angle_deg))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    lsg = lsg_mod()
    c = lsg.Context(0)
    yield c
    c.close()


def run_gpu(ctx, scan, p, range_only=False, tile=None):
    lsg = lsg_mod()
    if tile is not None:
        lsg.lsg_set_tile(ctx.h, tile)
    dev = torch.device("cuda", 0)
    elev = torch.from_numpy(scan.elev).to(dev)
    if range_only:
        out = ctx.segment(elev, range_=torch.from_numpy(scan.range).to(dev), az0=scan.az0, daz=scan.daz, params=p)
    else:
        out = ctx.segment(elev, xyzr=torch.from_numpy(scan.xyzr).to(dev), az0=scan.az0, daz=scan.daz, params=p)
    torch.cuda.synchronize()
    assert ctx.error() == lsg.LSG_OK
    if tile is not None:
        lsg.lsg_set_tile(ctx.h, lsg.TILES["16x240"])
    return (out.meshbits.cpu().numpy(), out.normals.cpu().numpy(), out.labels.cpu().numpy(),
            int(out.nseg.cpu()[0]))


def full_check(ctx, scan, p, range_only=False, tile=None, strict=True):
    mb, nrm, lab, nseg = run_gpu(ctx, scan, p, range_only, tile)
    rep = parity.check_outputs(ctx, scan, p, mb, nrm, lab, nseg, range_only=range_only, strict=strict)
    return rep, mb, nrm, lab, nseg


@pytest.mark.parametrize("make", [lidarsim.ring16, lidarsim.ring64, lidarsim.ring128],
                         ids=["ring16x1800", "ring64x2048_s2", "ring128x4096"])
def test_single_scan_workloads(ctx, make):
    spec = make()
    scan = lidarsim.make_scan(spec)
    rep, *_ = full_check(ctx, scan, params_of(spec))
    print(f"\n{spec.name}: {rep}")
    assert rep.vertices > 0


@pytest.mark.parametrize("make", [lidarsim.ring16, lidarsim.ring128],
                         ids=["ring16x1800", "ring128x4096"])
def test_auto_tile_equals_fixed(ctx, make):
    """LSG_TILE_AUTO picks a shape per call; the outputs do not depend on it."""
    lsg = lsg_mod()
    spec = make()
    scan = lidarsim.make_scan(spec)
    p = params_of(spec)
    lsg.lsg_set_tile(ctx.h, lsg.LSG_TILE_AUTO)
    auto = run_gpu(ctx, scan, p)
    lsg.lsg_set_tile(ctx.h, lsg.LSG_TILE_AUTO)
    for tile in ("32x240", "16x120", "8x120", "4x120", "2x120"):
        fixed = run_gpu(ctx, scan, p, tile=lsg.TILES[tile])
        for a, b in zip(auto, fixed):
            assert np.array_equal(a, b), tile
    with pytest.raises(lsg.LsgError):
        lsg.lsg_set_tile(ctx.h, lsg.LSG_TILE_COUNT)


def test_range_only_decode(ctx):
    spec = lidarsim.ring64(cols=1024)
    scan = lidarsim.make_scan(spec)
    rep, *_ = full_check(ctx, scan, params_of(spec), range_only=True)
    print(f"\nrange-only: {rep}")


def test_component_predicate(ctx):
    lsg = lsg_mod()
    spec = lidarsim.ring16()
    scan = lidarsim.make_scan(spec)
    rep, *_ = full_check(ctx, scan, params_of(spec, predicate=lsg.LSG_PRED_COMPONENT, comp=(0.2, 0.2, 0.2)))
    print(f"\ncomponent: {rep}")


RAGGED = [
    # (rings, cols, s, wrap, tile)
    (1, 1, 1, 1, "16x240"), (1, 7, 1, 1, "16x240"), (2, 2, 1, 1, "16x240"), (3, 3, 1, 1, "64x240"),
    (9, 131, 1, 1, "32x120"), (9, 131, 1, 0, "32x120"), (17, 257, 2, 1, "32x480"), (17, 257, 3, 0, "32x120"),
    (5, 1030, 1, 1, "32x240"), (33, 129, 1, 1, "64x240"), (16, 1800, 5, 1, "16x240"), (7, 1000, 15, 1, "32x480"),
    (64, 300, 1, 1, "32x120"), (3, 512, 2, 1, "32x240"), (24, 640, 4, 0, "64x240"),
    (8, 240, 1, 1, "16x240"), (8, 241, 1, 1, "16x240"), (5, 481, 1, 1, "32x480"), (3, 61, 1, 1, "32x120"),
    (35, 121, 1, 0, "32x120"), (17, 121, 1, 1, "16x120"), (33, 361, 2, 1, "16x120"), (16, 120, 1, 0, "16x120"),
    (9, 241, 1, 1, "8x120"), (8, 120, 3, 0, "8x120"), (25, 1800, 1, 1, "8x120"),
    (3, 130, 1, 1, "4x120"), (13, 483, 2, 0, "4x120"), (16, 1800, 1, 1, "4x120"),
    (3, 130, 1, 1, "2x120"), (13, 483, 2, 0, "2x120"), (7, 241, 1, 1, "2x120"), (16, 1800, 1, 1, "2x120"),
]


@pytest.mark.parametrize("H,W,s,wrap,tile", RAGGED)
def test_ragged_shapes(ctx, H, W, s, wrap, tile):
    lsg = lsg_mod()
    spec = lidarsim.ring64(seed=4000 + H * 31 + W, cols=W, rings=max(H, 2), subsample=s, angle_deg=10.0)
    spec = replace(spec, elev_deg=lidarsim.elev_horizon_dense(max(H, 2))[:H], p_drop=0.1)
    scan = lidarsim.make_scan(spec)
    full_check(ctx, scan, params_of(spec, wrap=wrap), tile=lsg.TILES[tile])


RANGE_RAGGED = [(17, 257, 3, 0, "4x120"), (9, 131, 1, 1, "8x120"), (33, 361, 2, 1, "16x120"),
                (5, 1030, 1, 1, "32x240"), (35, 121, 1, 0, "32x120"), (5, 361, 3, 1, "2x120")]


@pytest.mark.parametrize("H,W,s,wrap,tile", RANGE_RAGGED)
def test_range_only_ragged_shapes(ctx, H, W, s, wrap, tile):
    """Range-only decode (4-byte asynchronous copies, x,y,z formed when a
    row is read) on ragged shapes, small tiles and both seam modes."""
    lsg = lsg_mod()
    spec = lidarsim.ring64(seed=4400 + H * 31 + W, cols=W, rings=max(H, 2), subsample=s, angle_deg=10.0)
    spec = replace(spec, elev_deg=lidarsim.elev_horizon_dense(max(H, 2))[:H], p_drop=0.1)
    scan = lidarsim.make_scan(spec)
    full_check(ctx, scan, params_of(spec, wrap=wrap), range_only=True, tile=lsg.TILES[tile])


def test_edge_cases(ctx):
    lsg = lsg_mod()
    dev = torch.device("cuda", 0)
    p = lsg.Params()
    # empty scans
    for H, W in ((0, 0), (0, 16), (5, 0)):
        xyzr = torch.zeros((H, W, 4), device=dev)
        out = ctx.segment(torch.zeros(H, device=dev), xyzr=xyzr, daz=0.01, params=p)
        torch.cuda.synchronize()
        assert int(out.nseg.cpu()[0]) == 0
    # all dropouts
    spec = lidarsim.ring16(cols=256)
    scan = lidarsim.make_scan(spec)
    scan.xyzr[...] = 0
    mb, nrm, lab, nseg = run_gpu(ctx, scan, params_of(spec))
    assert nseg == 0 and (lab == -1).all() and (mb == 0).all()
    # one point
    one = lidarsim.Scan(spec, np.array([[[3.0, 0.0, 0.0, 3.0]]], np.float32), np.zeros((1, 1), np.int32),
                        np.zeros(1, np.float32), 0.0, 0.01)
    mb, nrm, lab, nseg = run_gpu(ctx, one, params_of(spec))
    assert nseg == 1 and lab[0, 0] == 0 and mb[0, 0] == lsg.BIT_VALID
    # bad arguments are refused synchronously
    bad = lsg.Params(subsample=0)
    with pytest.raises(lsg.LsgError) as ei:
        ctx.segment(torch.zeros(2, device=dev), xyzr=torch.zeros((2, 4, 4), device=dev), params=bad)
    assert ei.value.status == lsg.LSG_E_ARG
    with pytest.raises(lsg.LsgError):
        ctx.segment(torch.zeros(2, device=dev), xyzr=torch.zeros((2, 4, 4), device=dev),
                    params=lsg.Params(angle_rad=0.0))


def test_maximum_shapes(ctx):
    lsg = lsg_mod()
    # the longest ring the ABI accepts, and the most rings
    for H, W in ((1, 1 << 20), (4096, 16)):
        spec = lidarsim.ring16(seed=77, cols=W)
        spec = replace(spec, elev_deg=lidarsim.elev_uniform(-20, 5, H))
        scan = lidarsim.make_scan(spec)
        full_check(ctx, scan, params_of(spec))


def test_label_from_mask_random_masks(ctx):
    """Labels of random consistent masks (many tiles, seams, tile borders)."""
    rng = np.random.default_rng(99)
    dev = torch.device("cuda", 0)
    lsg = lsg_mod()
    for case in range(40):
        H = int(rng.integers(1, 40))
        W = int(rng.integers(1, 700))
        s = int(rng.integers(1, 4))
        wrap = int(rng.integers(0, 2))
        Ws = O.ws_of(W, s)
        p_h = rng.uniform(0.3, 0.97)
        valid_full = (rng.random((H, W)) < 0.85).astype(np.uint8)
        mb = np.zeros((H, Ws), np.uint8)
        vv = valid_full[:, ::s][:, :Ws] > 0
        mb[vv] |= O.BIT_VALID
        nb = parity.neighbour_index(H, Ws, wrap and Ws >= 3).reshape(-1, 3)
        flat = mb.ravel()
        for e, (eb, hb) in enumerate(((O.BIT_R, O.BIT_HR), (O.BIT_D, O.BIT_HD), (O.BIT_G, O.BIT_HG))):
            q = nb[:, e]
            ok = (q >= 0) & vv.ravel() & np.where(q >= 0, vv.ravel()[np.maximum(q, 0)], False)
            hom = ok & (rng.random(len(q)) < p_h)
            flat[ok] |= eb
            flat[hom] |= hb
        mb = flat.reshape(H, Ws)
        want, nwant = O.label_from_mask(mb, valid_full, W, s, wrap)
        for tile in ("16x240", "32x120", "32x480", "16x120", "8x120", "4x120", "2x120"):
            lsg.lsg_set_tile(ctx.h, lsg.TILES[tile])
            got, n = ctx.label_from_mask(torch.from_numpy(mb).to(dev), torch.from_numpy(valid_full).to(dev), W, s,
                                         wrap)
            torch.cuda.synchronize()
            assert np.array_equal(got.cpu().numpy(), want), (case, H, W, s, wrap, tile)
            assert int(n.cpu()[0]) == nwant
    lsg.lsg_set_tile(ctx.h, lsg.TILES["16x240"])


def test_nan_elevation_is_flagged_not_faulted(ctx):
    lsg = lsg_mod()
    spec = lidarsim.ring16(cols=128)
    scan = lidarsim.make_scan(spec)
    scan.elev[3] = np.nan
    dev = torch.device("cuda", 0)
    ctx.segment(torch.from_numpy(scan.elev).to(dev), xyzr=torch.from_numpy(scan.xyzr).to(dev), daz=scan.daz,
                params=params_of(spec))
    torch.cuda.synchronize()
    assert ctx.error() == lsg.LSG_E_DEVICE
    assert ctx.error() == lsg.LSG_OK  # the word is cleared by reading it


def test_budget_is_enforced(gpu_lib):
    lsg = lsg_mod()
    small = lsg.Context(0, budget_bytes=1 << 16)
    spec = lidarsim.ring128()
    scan = lidarsim.make_scan(spec)
    dev = torch.device("cuda", 0)
    with pytest.raises(lsg.LsgError) as ei:
        small.segment(torch.from_numpy(scan.elev).to(dev), xyzr=torch.from_numpy(scan.xyzr).to(dev),
                      daz=scan.daz, params=params_of(spec))
    assert ei.value.status == lsg.LSG_E_BUDGET
    small.close()

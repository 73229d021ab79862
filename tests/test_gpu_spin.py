"""Streaming (lsg_spin_*, Sec. 2: the mesh can be built while the sensor
acquires the scan): a revolution pushed column range by column range gives
lsg_segment's outputs bit for bit, and meets the oracle's parity bars on its
own.  Columns not yet pushed hold garbage, so a tile computed before its
columns arrived would show."""
import math
from dataclasses import replace

import numpy as np
import pytest

import lidarsim
import parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def mod():
    from paper_2005_02704_gb300 import lsg
    return lsg


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    lsg = mod()
    c = lsg.Context(0)
    yield c
    c.close()


def params_of(spec, wrap=1):
    lsg = mod()
    return lsg.Params(subsample=spec.subsample, r_max=spec.r_max, jump_rel_h=spec.jump_rel_h,
                      jump_rel_v=spec.jump_rel_v, angle_rad=math.radians(spec.angle_deg), wrap=wrap)


def schedule(W, n, rng):
    """n increasing cut points ending at W (repeats allowed)."""
    cuts = sorted(int(x) for x in rng.integers(0, W + 1, size=max(n - 1, 0)))
    return cuts + [W]


CASES = [
    ("ring16", lidarsim.ring16(cols=1800), 1, 16),
    ("ring64-s2", lidarsim.ring64(cols=2048), 1, 9),
    ("ring128", lidarsim.ring128(cols=1024), 1, 40),
    ("w257-s3-nowrap", replace(lidarsim.ring64(seed=91, cols=257, rings=17), subsample=3), 0, 7),
    ("w131-wrap", lidarsim.ring64(seed=92, cols=131, rings=9, subsample=1), 1, 131),
    ("w61", lidarsim.ring64(seed=93, cols=61, rings=3, subsample=1), 1, 5),
    ("w7-one-ring", replace(lidarsim.ring16(seed=94, cols=7), elev_deg=[-5.0]), 1, 3),
    ("w1030-one-push", lidarsim.ring64(seed=95, cols=1030, rings=5, subsample=1), 1, 1),
]


@pytest.mark.parametrize("tile", ["32x120", "16x240", "32x480", "16x120", "8x120", "4x120", "2x120"])
@pytest.mark.parametrize("name,spec,wrap,npush", CASES, ids=[c[0] for c in CASES])
def test_spin_equals_segment(ctx, name, spec, wrap, npush, tile):
    lsg = mod()
    lsg.lsg_set_tile(ctx.h, lsg.TILES[tile])
    dev = torch.device("cuda", 0)
    scan = lidarsim.make_scan(spec)
    p = params_of(spec, wrap)
    elev = torch.from_numpy(scan.elev).to(dev)
    full = torch.from_numpy(scan.xyzr).to(dev)
    want = ctx.segment(elev, xyzr=full, az0=scan.az0, daz=scan.daz, params=p)
    rng = np.random.default_rng(len(name) * 1000 + npush)
    buf = torch.from_numpy(rng.uniform(-30, 30, size=scan.xyzr.shape).astype(np.float32)).to(dev)
    buf[..., 3] = torch.from_numpy(rng.uniform(0.5, 60, size=scan.xyzr.shape[:2]).astype(np.float32)).to(dev)
    spin = lsg.Spin(ctx, elev, xyzr=buf, az0=scan.az0, daz=scan.daz, params=p)
    c0 = 0
    for c1 in schedule(scan.cols, npush, rng):
        buf[:, c0:c1] = full[:, c0:c1]
        spin.push(c1)
        c0 = c1
    got = spin.finish()
    torch.cuda.synchronize()
    assert ctx.error() == lsg.LSG_OK
    assert torch.equal(got.meshbits, want.meshbits)
    assert torch.equal(got.normals, want.normals)
    assert torch.equal(got.labels, want.labels)
    assert torch.equal(got.nseg, want.nseg)
    spin.close()
    lsg.lsg_set_tile(ctx.h, lsg.TILES["32x240"])


def stream_scan(ctx, scan, p, npush, seed, tile):
    """Pushes the scan into a garbage-filled buffer in npush column ranges and
    returns the finished outputs as numpy arrays."""
    lsg = mod()
    lsg.lsg_set_tile(ctx.h, lsg.TILES[tile])
    dev = torch.device("cuda", 0)
    elev = torch.from_numpy(scan.elev).to(dev)
    full = torch.from_numpy(scan.xyzr).to(dev)
    rng = np.random.default_rng(seed)
    buf = torch.from_numpy(rng.uniform(-30, 30, size=scan.xyzr.shape).astype(np.float32)).to(dev)
    spin = lsg.Spin(ctx, elev, xyzr=buf, az0=scan.az0, daz=scan.daz, params=p)
    c0 = 0
    for c1 in schedule(scan.cols, npush, rng):
        buf[:, c0:c1] = full[:, c0:c1]
        spin.push(c1)
        c0 = c1
    got = spin.finish()
    torch.cuda.synchronize()
    assert ctx.error() == lsg.LSG_OK
    spin.close()
    lsg.lsg_set_tile(ctx.h, lsg.TILES["32x240"])
    return (got.meshbits.cpu().numpy(), got.normals.cpu().numpy(), got.labels.cpu().numpy(),
            int(got.nseg.cpu()[0]))


ORACLE_CASES = [c for c in CASES if c[0] in ("ring16", "w257-s3-nowrap", "w131-wrap", "w61")]


@pytest.mark.parametrize("tile", ["32x120", "4x120"])
@pytest.mark.parametrize("name,spec,wrap,npush", ORACLE_CASES, ids=[c[0] for c in ORACLE_CASES])
def test_spin_meets_the_oracle(ctx, name, spec, wrap, npush, tile):
    scan = lidarsim.make_scan(spec)
    p = params_of(spec, wrap)
    mb, nrm, lab, nseg = stream_scan(ctx, scan, p, npush, 7 * npush + len(name), tile)
    rep = parity.check_outputs(ctx, scan, p, mb, nrm, lab, nseg)
    print(f"\nstreamed {name} ({tile}): {rep}")
    assert rep.vertices > 0


def test_spin_argument_errors(ctx):
    lsg = mod()
    dev = torch.device("cuda", 0)
    scan = lidarsim.make_scan(lidarsim.ring16(cols=600))
    elev = torch.from_numpy(scan.elev).to(dev)
    xyzr = torch.from_numpy(scan.xyzr).to(dev)
    spin = lsg.Spin(ctx, elev, xyzr=xyzr, az0=scan.az0, daz=scan.daz, params=params_of(lidarsim.ring16()))
    spin.push(300)
    with pytest.raises(lsg.LsgError):
        spin.push(200)                     # columns in place cannot decrease
    with pytest.raises(lsg.LsgError):
        spin.push(601)                     # past the last column
    spin.finish()
    with pytest.raises(lsg.LsgError):
        spin.finish()                      # finished once
    with pytest.raises(lsg.LsgError):
        spin.push(600)
    torch.cuda.synchronize()
    spin.close()
    # an empty revolution finishes with no segments
    e = torch.zeros((0, 5, 4), dtype=torch.float32, device=dev)
    spin = lsg.Spin(ctx, torch.zeros(0, device=dev), xyzr=e, params=lsg.Params())
    spin.push(0)
    out = spin.finish()
    torch.cuda.synchronize()
    assert int(out.nseg.item()) == 0
    spin.close()

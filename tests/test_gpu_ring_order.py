"""Ring order on the GPU (Sec. 2: rings from the topmost down, whatever order
the input rows come in; ties between equal elevations by input row).

A single-scan call of at most 256 rings finds the ring order inside its tile
kernel (a fast path for elevations that fall or rise strictly along the input
rows, a rank count otherwise); batched plans and larger scans take it from
k_prep.  The outputs are in ring order, so permuting a scan's input rows must
leave every output bit for bit unchanged, on both paths; scans with tied
elevations must meet the oracle.
"""
import math
from dataclasses import replace

import numpy as np
import pytest

import lidarsim
import parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def lsg_mod():
    from paper_2005_02704_gb300 import lsg
    return lsg


def params_of(spec):
    lsg = lsg_mod()
    return lsg.Params(subsample=spec.subsample, r_max=spec.r_max, jump_rel_h=spec.jump_rel_h,
                      jump_rel_v=spec.jump_rel_v, angle_rad=math.radians(spec.angle_deg))


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    lsg = lsg_mod()
    c = lsg.Context(0)
    yield c
    c.close()


def permuted(scan, perm):
    return lidarsim.Scan(scan.spec, np.ascontiguousarray(scan.xyzr[perm]), np.ascontiguousarray(scan.gt[perm]),
                         np.ascontiguousarray(scan.elev[perm]), scan.az0, scan.daz)


def segment(ctx, scan, p, tile):
    lsg = lsg_mod()
    lsg.lsg_set_tile(ctx.h, lsg.LSG_TILE_AUTO if tile == "auto" else lsg.TILES[tile])
    try:
        dev = torch.device("cuda", 0)
        out = ctx.segment(torch.from_numpy(scan.elev).to(dev), xyzr=torch.from_numpy(scan.xyzr).to(dev),
                          az0=scan.az0, daz=scan.daz, params=p)
        torch.cuda.synchronize()
        assert ctx.error() == lsg.LSG_OK
        return [t.cpu() for t in (out.meshbits, out.normals, out.labels, out.nseg)]
    finally:
        lsg.lsg_set_tile(ctx.h, lsg.LSG_TILE_AUTO)


SCANS = [
    ("ring16 (elevations rise along the rows)", lidarsim.ring16(cols=600)),
    ("ring64 s=2 (elevations fall along the rows)", lidarsim.ring64(cols=512)),
    ("ring128 (rise)", lidarsim.ring128(cols=256)),
    ("300 rings (k_prep path)", replace(lidarsim.ring16(seed=71, cols=96), elev_deg=lidarsim.elev_uniform(-25, 15, 300))),
]


@pytest.mark.parametrize("tile", ["auto", "32x120", "2x120"])
@pytest.mark.parametrize("name,spec", SCANS, ids=[s[0].split(" ")[0] for s in SCANS])
def test_input_row_order_does_not_change_the_outputs(ctx, name, spec, tile):
    scan = lidarsim.make_scan(spec)
    p = params_of(spec)
    want = segment(ctx, scan, p, tile)
    H = scan.rings
    rng = np.random.default_rng(H * 7 + len(tile))
    for perm in (np.arange(H)[::-1], rng.permutation(H)):
        got = segment(ctx, permuted(scan, perm), p, tile)
        for a, b in zip(got, want):
            assert torch.equal(a, b), name


def test_tied_elevations_meet_the_oracle(ctx):
    """Pairs of rings at equal elevations, rows shuffled: the ring order breaks
    the ties by input row on the GPU as in the oracle (both single-scan paths:
    20 rings in the tile kernel, 280 through k_prep)."""
    for H, W, seed in ((20, 700, 81), (280, 64, 82)):
        elev = np.repeat(lidarsim.elev_uniform(-20, 8, H // 2), 2)
        spec = replace(lidarsim.ring16(seed=seed, cols=W), elev_deg=list(elev))
        scan = lidarsim.make_scan(spec)
        scan = permuted(scan, np.random.default_rng(seed).permutation(H))
        p = params_of(spec)
        mb, nrm, lab, nseg = (t.numpy() for t in segment(ctx, scan, p, "auto"))
        rep = parity.check_outputs(ctx, scan, p, mb, nrm, lab, int(nseg[0]))
        print(f"\n{H} rings in tied pairs: {rep}")

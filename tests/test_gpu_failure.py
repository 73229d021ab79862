"""Failure detection without a GPU fault: the persistent schedule's bounded
wait, run on a counter that nothing increments, gives up after a short limit
and flags a timeout that the host reads; the context stays usable."""
import math

import pytest

import lidarsim

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_bounded_wait_times_out_and_context_stays_usable(gpu_lib):
    from paper_2005_02704_gb300 import lsg
    lib = lsg.load()
    ctx = lsg.Context(0)
    dev = torch.device("cuda", 0)
    spec = lidarsim.ring16(cols=600)
    scan = lidarsim.make_scan(spec)
    p = lsg.Params(r_max=spec.r_max, angle_rad=math.radians(spec.angle_deg))
    elev = torch.from_numpy(scan.elev).to(dev)
    xyzr = torch.from_numpy(scan.xyzr).to(dev)
    want = ctx.segment(elev, xyzr=xyzr, az0=scan.az0, daz=scan.daz, params=p)
    torch.cuda.synchronize()
    assert ctx.error() == lsg.LSG_OK
    for _ in range(2):  # the timeout is reported, then cleared
        assert lib.lsg_selftest_wait_timeout(ctx.h) == lsg.LSG_OK
        assert ctx.error() == lsg.LSG_OK
    got = ctx.segment(elev, xyzr=xyzr, az0=scan.az0, daz=scan.daz, params=p)
    torch.cuda.synchronize()
    assert ctx.error() == lsg.LSG_OK
    assert torch.equal(got.labels, want.labels) and torch.equal(got.nseg, want.nseg)
    ctx.close()

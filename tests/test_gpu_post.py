"""GPU parity of the post-processing (Sec. 2, last paragraph): segment sizes,
small-segment removal and segment normal sums against the oracle, computed
on the same labels."""
import math

import numpy as np
import pytest

import lidarsim
import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("make,min_points", [(lidarsim.ring16, 5), (lidarsim.ring64, 3), (lidarsim.ring128, 20)],
                         ids=["ring16", "ring64_s2", "ring128"])
def test_segment_stats_match_oracle(gpu_lib, make, min_points):
    from paper_2005_02704_gb300 import lsg
    spec = make()
    scan = lidarsim.make_scan(spec)
    p = lsg.Params(subsample=spec.subsample, r_max=spec.r_max, jump_rel_h=spec.jump_rel_h,
                   jump_rel_v=spec.jump_rel_v, angle_rad=math.radians(spec.angle_deg))
    dev = torch.device("cuda", 0)
    ctx = lsg.Context(0)
    out = ctx.segment(torch.from_numpy(scan.elev).to(dev), xyzr=torch.from_numpy(scan.xyzr).to(dev), az0=scan.az0,
                      daz=scan.daz, params=p)
    torch.cuda.synchronize()
    labels_in = out.labels.cpu().numpy()
    normals = out.normals.cpu().numpy().astype(np.float64)
    mb = out.meshbits.cpu().numpy()
    sizes, nsum, nseg = ctx.segment_stats(out, scan.cols, spec.subsample, min_points, normal_sums=True)
    torch.cuda.synchronize()
    want_lab, want_sizes, want_nsum, want_kept = O.segment_stats(labels_in, min_points, s=spec.subsample,
                                                                 normals=normals, meshbits=mb)
    assert np.array_equal(out.labels.cpu().numpy(), want_lab)
    assert np.array_equal(sizes.cpu().numpy(), want_sizes)
    assert int(nseg.cpu()[0]) == want_kept
    got = nsum.cpu().numpy().astype(np.float64)
    # float32 recursive sum (any order) of at most n terms of magnitude <= 1:
    # |error| <= (n - 1) u sum|x| <= n (n - 1) u per component, u = 2^-24,
    # plus the float32 rounding of the normals themselves (n u)
    n = want_sizes.astype(np.float64)[:, None]
    assert np.all(np.abs(got - want_nsum) <= (n * n) * 2.0 ** -24 + 1e-6)
    assert want_kept < int(np.sum(want_sizes > 0)) or min_points <= 1  # something was removed
    ctx.close()


def test_min_points_zero_keeps_everything(gpu_lib):
    from paper_2005_02704_gb300 import lsg
    spec = lidarsim.ring16(cols=512)
    scan = lidarsim.make_scan(spec)
    dev = torch.device("cuda", 0)
    ctx = lsg.Context(0)
    out = ctx.segment(torch.from_numpy(scan.elev).to(dev), xyzr=torch.from_numpy(scan.xyzr).to(dev), daz=scan.daz,
                      params=lsg.Params(r_max=spec.r_max))
    before = out.labels.clone()
    n0 = int(out.nseg.cpu()[0])
    sizes, _, nseg = ctx.segment_stats(out, scan.cols, 1, 0)
    torch.cuda.synchronize()
    assert torch.equal(before, out.labels) and int(nseg.cpu()[0]) == n0
    assert int(sizes.sum().cpu()) == int((before >= 0).sum().cpu())
    ctx.close()

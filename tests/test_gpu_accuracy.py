"""The paper's accuracy protocol (Sec. 3, Table 2) run on the CUDA path.

Synthetic Velodyne-32E-like scenes (32 rings x 1800 shots, primitives on a
flat floor) stand in for the paper's Blensor dataset; the ground truth is the
primitive face each ray hit.  Segmentation uses the paper's component
predicate (I = J = K = 0.2) at sampling intervals 5, 10 and 15.  The paper
reports accuracy falling as the interval grows (its Table 2, through
precision); the test checks that trend and that every score is a proper
fraction, and checks one of the scans against the oracle's parity bars with
the same predicate.  The scores are printed.
"""
import math

import numpy as np
import pytest

import lidarsim
import parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_table2_protocol_on_synthetic_scenes(gpu_lib):
    from paper_2005_02704_gb300 import evaluate
    rows = evaluate.table2(n_scenes=2)
    print("\ninterval  precision  recall  F1")
    for s, p, r, f in rows:
        print(f"{s:8d}  {p:9.4f}  {r:6.4f}  {f:.4f}")
    assert [r[0] for r in rows] == [5, 10, 15]
    for _, p, r, f in rows:
        assert 0.0 < p <= 1.0 and 0.0 < r <= 1.0 and 0.0 < f <= 1.0
        assert math.isclose(f, 2 * p * r / (p + r), rel_tol=0.2)  # a mean of F1s, near the F1 of the means
    f1 = [r[3] for r in rows]
    prec = [r[1] for r in rows]
    assert f1[0] > f1[1] > f1[2]
    assert prec[0] > prec[1] > prec[2]


@pytest.mark.parametrize("s", [5, 15])
def test_table2_scene_meets_the_oracle(gpu_lib, s):
    from paper_2005_02704_gb300 import evaluate, lsg
    spec = evaluate.velodyne32_scene(4000)
    scan = lidarsim.make_scan(spec)
    p = lsg.Params(subsample=s, r_max=spec.r_max, jump_rel_h=spec.jump_rel_h, jump_rel_v=spec.jump_rel_v,
                   predicate=lsg.LSG_PRED_COMPONENT, angle_rad=math.radians(10.0), comp=(0.2, 0.2, 0.2))
    ctx = lsg.Context(0)
    dev = torch.device("cuda", 0)
    out = ctx.segment(torch.from_numpy(scan.elev).to(dev), xyzr=torch.from_numpy(scan.xyzr).to(dev),
                      az0=scan.az0, daz=scan.daz, params=p)
    torch.cuda.synchronize()
    assert ctx.error() == lsg.LSG_OK
    rep = parity.check_outputs(ctx, scan, p, out.meshbits.cpu().numpy(), out.normals.cpu().numpy(),
                               out.labels.cpu().numpy(), int(out.nseg.cpu()[0]))
    ctx.close()
    print(f"\nvelodyne32 s={s}: {rep}")
    assert rep.vertices > 0 and np.isfinite(rep.max_err_well)

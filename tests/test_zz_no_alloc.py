"""The allocation-free entry point, lsg_segment_noalloc, against lsg_segment.

Some callers cannot call cudaMalloc: a sensor thread with a hard latency
budget (allocation can synchronise the device and take driver-wide locks) or
a host framework that owns all device memory.  lsg_segment_noalloc keeps its
workspace in a fixed device array inside the library instead.  This test
calls it through the C ABI twice in a row, on scans of different shapes (the
second call finds the first call's leftovers in the shared array), and checks
each result against lsg_segment on the same inputs with the tolerances the
other GPU tests use: mesh bits, labels and segment count exact, normals
within 1e-4 rad.  It also checks that a scan beyond the array's capacity is
refused before anything is launched, and that a NaN elevation (bad input the
device sees) is reported by lsg_noalloc_get_error, which also allocates
nothing, and cleared by reading it.

The file name makes pytest collect it last; it creates its own context and
inputs, so it also passes alone in a fresh process.
"""
import math

import numpy as np
import pytest

import lidarsim

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _params(spec):
    from paper_2005_02704_gb300 import lsg
    return lsg.Params(subsample=spec.subsample, r_max=spec.r_max, jump_rel_h=spec.jump_rel_h,
                      jump_rel_v=spec.jump_rel_v, angle_rad=math.radians(spec.angle_deg))


def _angle(a, b):
    cr = np.cross(a, b)
    return np.arctan2(np.linalg.norm(cr, axis=-1), np.sum(a * b, axis=-1))


def test_noalloc_matches_lsg_segment_on_two_calls_in_a_row(gpu_lib):
    from paper_2005_02704_gb300 import lsg
    dev = torch.device("cuda", 0)
    ctx = lsg.Context(0)
    specs = [lidarsim.ring128(), lidarsim.ring64()]  # 524,288 then 65,536 vertices (s = 2)
    for spec in specs:
        scan = lidarsim.make_scan(spec)
        p = _params(spec)
        elev = torch.from_numpy(scan.elev).to(dev)
        xyzr = torch.from_numpy(scan.xyzr).to(dev)
        want = ctx.segment(elev, xyzr=xyzr, az0=scan.az0, daz=scan.daz, params=p)
        got = lsg.alloc_outputs(scan.rings, scan.cols, p.subsample, dev)
        got.meshbits.fill_(0xAA)
        got.labels.fill_(-7)
        st = lsg.lsg_segment_noalloc(lsg.make_scan(elev, xyzr, None, scan.az0, scan.daz), p.to_c(), got.to_c(),
                                     torch.cuda.current_stream().cuda_stream)
        assert st == lsg.LSG_OK, lsg.lsg_status_str(st)
        torch.cuda.synchronize()
        assert torch.equal(got.meshbits, want.meshbits)
        assert torch.equal(got.labels, want.labels)
        assert int(got.nseg.cpu()[0]) == int(want.nseg.cpu()[0])
        has = (want.meshbits.cpu().numpy() & lsg.BIT_HASN) > 0
        a = got.normals.cpu().numpy()[has].astype(np.float64)
        b = want.normals.cpu().numpy()[has].astype(np.float64)
        assert has.any() and _angle(a, b).max() <= 1e-4
    ctx.close()


def test_noalloc_refuses_scans_beyond_its_fixed_workspace(gpu_lib):
    from paper_2005_02704_gb300 import lsg
    dev = torch.device("cuda", 0)
    H, W = 512, 4096  # 2,097,152 vertices > LSG_NOALLOC_MAX_VERTICES
    assert H * W > lsg.LSG_NOALLOC_MAX_VERTICES
    elev = torch.zeros(H, device=dev)
    xyzr = torch.zeros((H, W, 4), device=dev)
    out = lsg.alloc_outputs(H, W, 1, dev)
    st = lsg.lsg_segment_noalloc(lsg.make_scan(elev, xyzr, None, 0.0, 2 * math.pi / W), lsg.Params().to_c(),
                                 out.to_c(), torch.cuda.current_stream().cuda_stream)
    assert st == lsg.LSG_E_SHAPE


def test_noalloc_reports_device_flags_through_its_error_query(gpu_lib):
    from paper_2005_02704_gb300 import lsg
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream().cuda_stream
    spec = lidarsim.ring16(cols=128)
    scan = lidarsim.make_scan(spec)
    p = _params(spec)
    xyzr = torch.from_numpy(scan.xyzr).to(dev)
    out = lsg.alloc_outputs(scan.rings, scan.cols, p.subsample, dev)
    good = torch.from_numpy(scan.elev).to(dev)
    bad = good.clone()
    bad[3] = float("nan")
    st = lsg.lsg_segment_noalloc(lsg.make_scan(bad, xyzr, None, scan.az0, scan.daz), p.to_c(), out.to_c(), stream)
    assert st == lsg.LSG_OK
    assert lsg.lsg_noalloc_get_error(stream) == lsg.LSG_E_DEVICE
    assert lsg.lsg_noalloc_get_error(stream) == lsg.LSG_OK  # cleared by reading it
    st = lsg.lsg_segment_noalloc(lsg.make_scan(good, xyzr, None, scan.az0, scan.daz), p.to_c(), out.to_c(), stream)
    assert st == lsg.LSG_OK
    assert lsg.lsg_noalloc_get_error(stream) == lsg.LSG_OK

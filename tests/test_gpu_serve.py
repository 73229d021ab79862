"""GPU tests of the serving path: every scan's result is the same alone and
in the continuous-batching mix (labels, segment count and mesh bytes exact,
normals within 1e-4 rad), also under a memory budget that forces admission to
wait."""
import numpy as np
import pytest

import lidarsim

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _alone_results(feeds):
    from paper_2005_02704_gb300 import lsg
    dev = torch.device("cuda", 0)
    ctx = lsg.Context(0)
    res = {}
    for f in feeds:
        for m, x in enumerate(f.host_xyzr):
            out = ctx.segment(f.host_elev.to(dev), xyzr=x.to(dev), az0=f.az0, daz=f.daz, params=f.params)
            torch.cuda.synchronize()
            res[(f.sensor, m)] = (out.labels.cpu(), int(out.nseg.cpu()[0]), out.meshbits.cpu(), out.normals.cpu())
    ctx.close()
    return res


def _check(reqs, feeds, alone):
    for r in reqs:
        m = r.ticket % len(feeds[r.sensor].host_xyzr)
        lab, nseg, mb, nrm = alone[(r.sensor, m)]
        assert torch.equal(r.result["labels"], lab), r.ticket
        assert r.result["nseg"] == nseg
        assert torch.equal(r.result["meshbits"], mb)
        a = r.result["normals"].double().numpy().reshape(-1, 3)
        b = nrm.double().numpy().reshape(-1, 3)
        has = (mb.numpy().reshape(-1) & 0x80) > 0
        cr = np.linalg.norm(np.cross(a[has], b[has]), axis=1)
        assert np.all(np.arctan2(cr, np.sum(a[has] * b[has], axis=1)) <= 1e-4)


@pytest.mark.parametrize("budget_mb,lanes,max_batch", [(1024, 3, 16), (60, 2, 4)])
def test_results_are_the_same_alone_and_in_the_mix(gpu_lib, budget_mb, lanes, max_batch):
    from paper_2005_02704_gb300 import serve
    feeds = serve.make_feeds(lidarsim.sensor_specs(8), scans_per_sensor=2)
    alone = _alone_results(feeds)
    trace = serve.arrival_trace([f.rate_hz for f in feeds], duration_s=3.0, burst=(1.0, 2.0, 4.0), seed=5)
    budget = budget_mb << 20
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    torch.cuda.reset_peak_memory_stats()
    server = serve.Server(budget_bytes=budget, lanes=lanes, max_batch=max_batch)
    stats = serve.run_served(server, feeds, trace, time_scale=10.0, keep_geometry=True)
    assert stats["scans"] == len(trace) == len(server.done)
    # the device footprint stays within the budget: the lanes' contexts (which
    # did not grow) plus the slots, whose tensors are the only torch
    # allocations the server makes
    assert sum(c.memory_used() for c in server.ctxs) == server.fixed_bytes
    assert server.fixed_bytes + server.pool.peak <= budget
    assert torch.cuda.max_memory_allocated() - base <= server.pool.budget
    assert max(server.batch_sizes) > 1  # scans were batched together
    _check(server.done, feeds, alone)
    server.close()


def test_serial_loop_runs(gpu_lib):
    from paper_2005_02704_gb300 import serve
    feeds = serve.make_feeds(lidarsim.sensor_specs(4), scans_per_sensor=1)
    trace = serve.arrival_trace([f.rate_hz for f in feeds], duration_s=0.5, burst=None, seed=2)
    stats = serve.run_serial(feeds, trace, time_scale=1e9)
    assert stats["scans"] == len(trace) and stats["p99_ms"] > 0

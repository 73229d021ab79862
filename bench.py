#!/usr/bin/env python
"""Benchmark of the Lidar surface-segmentation path on GB300.

Workload (per rank): 512 seeded ray-cast scans with rings drawn from
{16, 32, 64, 128} and widths from {1024, 1800, 2048, 4096} (about 69 M points,
1.1 GB of x,y,z,r input), sub-sampling 1, angle threshold 10 deg.  One step is
one batched pass over the whole batch (a CUDA-graph replay of the four
kernels) with inputs resident in HBM.  Inputs are larger than L2, so no flush
is needed between steps.

The JSON line reports points/s of the batched path (value), the same metric
end to end through the C ABI with host buffers (e2e: lsg_batch_plan_io, one
graph replay per step that copies the inputs from pinned host memory, runs
the pass and copies every output back, in chunks whose copies overlap the
other chunks' passes; the one-chunk variant and the host link's floor for the
same bytes are reported beside it), the plain
per-scan path (one lsg_segment call per scan), the dominant kernel's HBM
roofline fraction, and the FP64 oracle timed on the host cores on a bounded
sample (cpu_baseline).

Multi-GPU: scans are independent, so N ranks each segment their own batch
(weak scaling, no collective on the data path); timing is the max over ranks.

``--impl reference`` times the FP64 oracle on the host cores instead (the
reference arm: bounded samples of the same workload, same metric).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "points/sec segmented + p50/p99 scan latency, batched/served vs plain GPU"
UNIT = "points/s"
WORKLOAD = ("batch512: 512 seeded ray-cast Lidar scans per GPU, rings {16,32,64,128} x columns "
            "{1024,1800,2048,4096}, x,y,z,r float32 input, s=1, angle 10 deg, one CUDA-graph pass per step")
FALLBACK_HBM_GBS = 6800.0
# algorithmic bytes at s = 1: the pass reads x,y,z,r (16 B) per point and
# writes labels (4 B) per point plus a mesh byte and a normal (13 B) per
# vertex, and reads the range once more for validity (4 B): 8 + 25/s
PATH_BYTES_PER_POINT = 33.0
# the fused tile kernel alone: 16 B read, 13 B written per point (s = 1)
TILE_BYTES_PER_POINT = 29.0
# range-only input at s = 1: the range (4 B) and the labels (4 B) per point,
# a mesh byte and a normal (13 B) per vertex: 8 + 13/s
RANGE_PATH_BYTES_PER_POINT = 21.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["lsg", "reference"], default="lsg")
    ap.add_argument("--scans", type=int, default=512)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-generator", action="store_true", help="skip timing the GPU scan generator")
    ap.add_argument("--no-spin", action="store_true", help="skip the streaming (per-packet) latency measurement")
    ap.add_argument("--no-single", action="store_true", help="skip the single-scan latency measurement")
    ap.add_argument("--no-range-input", action="store_true", help="skip the range-only input measurement")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the Table-2 accuracy protocol")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffer) measurements")
    ap.add_argument("--no-schedules", action="store_true", help="skip timing every schedule of the plan")
    ap.add_argument("--single-only", action="store_true",
                    help="only the single-scan latency measurement (one JSON object; for profiling the per-call path)")
    ap.add_argument("--phased", action="store_true", help="force four phased launches (else the autotuner's choice)")
    ap.add_argument("--fused", action="store_true", help="force the single persistent launch")
    ap.add_argument("--grouped", action="store_true", help="force the grouped schedule")
    ap.add_argument("--e2e-chunks", type=int, default=16, help="chunks of the pipelined end-to-end path")
    ap.add_argument("--tile", default=None, help="force a tile shape (e.g. 32x240) instead of autotuning")
    ap.add_argument("--serve-scale", type=float, default=10.0,
                    help="time compression of the 60 s sensor trace for the served measurement")
    return ap.parse_args()


def dist_env():
    from paper_2005_02704_gb300 import replicas
    return replicas.env()


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for k, nm in enumerate(names):
                    if f[5 + k].lower().startswith("active"):
                        reasons.add(nm)
            os.unlink(self.path)
        except Exception:
            return None
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# --------------------------------------------------------------------------
# helpers
# --------------------------------------------------------------------------
def measured_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


SCHEDULES = {0: "phased (4 launches)", 1: "fused (one persistent launch)",
             2: "grouped (ring order, then 4 scan groups of tile / merge / label launches on parallel graph branches)"}


def kernel_code_digest() -> str:
    """SHA-256 of the kernels' code: lsg_kernels.cu with its comments, trailing
    blanks and empty lines removed (the file has no comment markers inside
    string literals), so that editing a comment keeps a capture valid."""
    src = os.path.join(ROOT, "paper_2005_02704_gb300", "csrc", "lsg_kernels.cu")
    text = re.sub(r"/\*.*?\*/", "", open(src).read(), flags=re.S)
    lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines()]
    return hashlib.sha256("\n".join(ln for ln in lines if ln).encode()).hexdigest()


def profiled_values(profile: str):
    """The machine-readable lines (- key: `value`) of a committed ncu summary
    under profiles/, or None when the kernels' code has changed since the
    capture (the summary's kernel_source_sha256, kernel_code_digest() at the
    time, no longer matches)."""
    prof = os.path.join(ROOT, "profiles", profile)
    try:
        sha = kernel_code_digest()
        vals = {}
        for line in open(prof):
            if ":" in line and line.strip().startswith("- "):
                k, v = line.strip()[2:].split(":", 1)
                vals[k.strip()] = v.strip().strip("`")
        if vals.get("kernel_source_sha256") != sha:
            return None
        return vals
    except Exception:
        return None


def profiled_traffic(kernel: str):
    """DRAM bytes per point of the kernel from its committed ncu summary,
    valid only while the kernel source is unchanged since the capture."""
    vals = profiled_values(f"{kernel}_batch512.md")
    try:
        return float(vals["dram_bytes_per_point"]) if vals else None
    except (KeyError, ValueError):
        return None


def batch_data(n, rank):
    import lidarsim
    from paper_2005_02704_gb300 import replicas
    specs = lidarsim.batch_specs(n, seed0=replicas.shard_seed0(rank, n))
    scans = [lidarsim.make_scan(sp) for sp in specs]
    return specs, scans


def seg_params(spec):
    from paper_2005_02704_gb300 import lsg
    return lsg.Params(subsample=spec.subsample, r_max=spec.r_max, jump_rel_h=spec.jump_rel_h,
                      jump_rel_v=spec.jump_rel_v, angle_rad=math.radians(spec.angle_deg))


def oracle_rate(specs, scans, budget_points, threads):
    """FP64 oracle over a bounded sample of the batch on the host cores."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle as O
    stride = max(1, int(math.ceil(sum(s.points for s in scans) / budget_points)))
    idx = list(range(0, len(scans), stride))
    pts = sum(scans[i].points for i in idx)

    def one(i):
        sp = specs[i]
        p = O.Params(subsample=sp.subsample, r_max=sp.r_max, jump_rel_h=sp.jump_rel_h, jump_rel_v=sp.jump_rel_v,
                     angle_rad=math.radians(sp.angle_deg))
        O.segment_scan(scans[i], p)

    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(one, idx))
    dt = time.perf_counter() - t0
    return pts / dt, pts, len(idx), dt


def workload_config(n_scans, points, world):
    """The workload both arms measure (identical dicts on both arms)."""
    return {"workload": WORKLOAD, "scans_per_gpu": n_scans, "points_per_gpu": points,
            "l2": "inputs larger than L2 (x,y,z,r %.2f GB per GPU > 129 MB), no flush" % (points * 16 / 1e9),
            "parallelism": f"replicas x{world}"}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# --------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# --------------------------------------------------------------------------
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    specs, scans = batch_data(args.scans, 0)
    cores = host_cores()
    points = sum(s.points for s in scans)
    # each step is the whole batch, one scan per thread on every host core
    # (about a second of host work per step at 16 cores)
    for _ in range(args.warmup):
        oracle_rate(specs, scans, float(points), cores)
    pts_total, t_total = 0, 0.0
    for _ in range(args.steps):
        r, pts, ns, dt = oracle_rate(specs, scans, float(points), cores)
        pts_total += pts
        t_total += dt
    value = pts_total / t_total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(len(scans), points, args.gpus),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"the whole batch ({len(scans)} scans, {points / 1e6:.1f} M points) per step, "
                                       f"one scan per thread on {cores} threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# served path
# --------------------------------------------------------------------------
def serve_measurement(args, local, world, max_over_ranks, sum_over_ranks):
    """8 simulated sensors (rings {16,32,64,128}, two each; 10-20 Hz Poisson
    arrivals; 4x burst over [30, 40) s) for 60 s of simulated time, replayed
    --serve-scale times faster than real time, on an 8 GB admission budget.
    Reports p50/p99 arrival-to-results-on-host latency and scans/s for the
    continuous-batching server and for the serial plain-kernel loop on the
    same trace, plus both at saturation (all arrivals at once)."""
    import lidarsim
    from paper_2005_02704_gb300 import serve
    feeds = serve.make_feeds(lidarsim.sensor_specs(8, seed0=3000 + 8 * int(os.environ.get("RANK", "0"))),
                             scans_per_sensor=4)
    trace = serve.arrival_trace([f.rate_hz for f in feeds], duration_s=60.0, burst=(30.0, 40.0, 4.0), seed=17)
    scale = args.serve_scale
    server = serve.Server(budget_bytes=8 << 30, lanes=3, max_batch=64, device=local)
    sat_n = min(len(trace), 4000)
    serve.run_served(server, feeds, trace[:sat_n], float("inf"))  # warm-up: slots for the deepest queue
    k0 = len(server.batch_sizes)
    saturated = serve.run_served(server, feeds, trace[:sat_n], float("inf"))
    k1 = len(server.batch_sizes)
    nominal = serve.run_served(server, feeds, trace, scale)
    pool_peak = server.pool.peak
    sat_sizes, nom_sizes = server.batch_sizes[k0:k1], server.batch_sizes[k1:]
    server.close()
    serve.run_serial(feeds, trace[:50], float("inf"), device=local)  # warm-up
    serial = serve.run_serial(feeds, trace, scale, device=local)
    serial_sat = serve.run_serial(feeds, trace[:sat_n], float("inf"), device=local)

    def agg(d):
        return {"p50_ms": max_over_ranks(d["p50_ms"]), "p99_ms": max_over_ranks(d["p99_ms"]),
                "scans_per_s": sum_over_ranks(d["scans_per_s"]), "points_per_s": sum_over_ranks(d["points_per_s"]),
                "scans": int(sum_over_ranks(d["scans"])),
                # this rank's sensors (the shapes differ between ranks): no reduction
                "p50_ms_by_shape": d["p50_ms_by_shape"]}

    def batches(sizes):
        return {"batches": len(sizes), "mean_batch": float(sum(sizes) / max(1, len(sizes))),
                "share_of_one": float(sum(1 for x in sizes if x == 1) / max(1, len(sizes)))}

    return {"trace": f"8 sensors, 60 s simulated at {scale:g}x real time, {len(trace)} scans per GPU, "
                     "10-20 Hz Poisson + 4x burst [30,40) s, 8 GB admission budget, 3 lanes, batch <= 64",
            "batched": agg(nominal), "serial_plain": agg(serial),
            "saturated": {"batched": agg(saturated), "serial_plain": agg(serial_sat), "scans": sat_n},
            "p99_gain": serial["p99_ms"] / max(nominal["p99_ms"], 1e-9),
            "throughput_gain_saturated": saturated["scans_per_s"] / max(serial_sat["scans_per_s"], 1e-9),
            "pool_peak_bytes": pool_peak, "batching": batches(nom_sizes), "batching_saturated": batches(sat_sizes)}


def generator_measurement(specs, local, steps, warmup, max_over_ranks, sum_over_ranks):
    """The GPU scan generator (lsg_raycast) producing the whole batch: one
    launch per scan into a scratch buffer, timed with CUDA events."""
    import numpy as np
    import torch

    import lidarsim
    from paper_2005_02704_gb300 import lsg
    dev = torch.device("cuda", local)
    jobs, total = [], 0
    for sp in specs:
        elev = torch.tensor([math.radians(e) for e in sp.elev_deg], dtype=torch.float32, device=dev)
        prims = torch.from_numpy(lidarsim.scene_prims(sp)).to(dev)
        jobs.append((sp, elev, prims, total))
        total += sp.rings * sp.cols
    xyzr = torch.empty((total, 4), dtype=torch.float32, device=dev)
    gt = torch.empty(total, dtype=torch.int32, device=dev)

    def once():
        for sp, elev, prims, off in jobs:
            n = sp.rings * sp.cols
            lsg.raycast(elev, sp.cols, float(np.float32(sp.az0)), float(np.float32(sp.daz)), prims, sp.sigma,
                        sp.p_drop, sp.r_max, sp.seed, xyzr=xyzr[off:off + n].view(sp.rings, sp.cols, 4),
                        gt=gt[off:off + n].view(sp.rings, sp.cols))

    for _ in range(warmup):
        once()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        once()
    e1.record()
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1) / steps)
    return {"path": "lsg_raycast, one launch per scan (the batch's scenes, rays and noise)",
            "ms_per_batch": ms, "rays_per_s": sum_over_ranks(total) / (ms / 1e3), "launches_per_batch": len(jobs)}


SINGLE_SCANS = (("ring16x1800", "ring16"), ("ring64x2048_s2", "ring64"), ("ring128x4096", "ring128"))


def pct(sorted_vals, q):
    """q-quantile of sorted values (nearest rank)."""
    return sorted_vals[min(len(sorted_vals) - 1, max(0, int(math.ceil(q * len(sorted_vals))) - 1))]


def single_scan_measurement(local, peak, reps=100, warm=10):
    """The three single-scan workloads (16 x 1800; 64 x 2048 at s = 2;
    128 x 4096) through lsg_segment, tile shape chosen per call: device
    latency of each of `reps` back-to-back calls (events around each call on
    the launching stream), p50 / p99, points/s at the median and the path's
    algorithmic bytes (8 + 25/s per point) against HBM.  Each scan (at most
    8.4 MB of input) stays resident in the 129 MB L2 between calls."""
    import torch

    import lidarsim
    from paper_2005_02704_gb300 import lsg
    dev = torch.device("cuda", local)
    ctx = lsg.Context(local)
    stream = torch.cuda.current_stream()
    res = {}
    for name, maker in SINGLE_SCANS:
        spec = getattr(lidarsim, maker)()
        scan = lidarsim.make_scan(spec)
        p = seg_params(spec)
        elev = torch.from_numpy(scan.elev).to(dev)
        xyzr = torch.from_numpy(scan.xyzr).to(dev)
        out = lsg.alloc_outputs(scan.rings, scan.cols, spec.subsample, dev)

        def call():
            ctx.segment(elev, xyzr=xyzr, az0=scan.az0, daz=scan.daz, params=p, out=out, stream=stream)

        for _ in range(warm):
            call()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        torch.cuda.synchronize()
        for a, b in ev:
            a.record(stream)
            call()
            b.record(stream)
        torch.cuda.synchronize()
        if ctx.error() != lsg.LSG_OK:
            raise RuntimeError("device error in the single-scan measurement")
        t = sorted(a.elapsed_time(b) for a, b in ev)
        p50, p99 = pct(t, 0.5), pct(t, 0.99)
        n = scan.rings * scan.cols
        bpp = 8.0 + 25.0 / spec.subsample
        res[name] = {"points": n, "subsample": spec.subsample, "p50_ms": p50, "p99_ms": p99,
                     "points_per_s": n / (p50 / 1e3), "scans_per_s": 1e3 / p50, "bytes_per_point": bpp,
                     "achieved_gbs": bpp * n / (p50 / 1e3) / 1e9,
                     "hbm_frac": bpp * n / (p50 / 1e3) / 1e9 / peak}
        res[name]["host_io"] = host_io_latency(ctx, scan, p, local, reps, warm)
    ctx.close()
    res["note"] = (f"{reps} back-to-back lsg_segment calls per scan after {warm} warm-up calls, tile shape per call; "
                   "L2-resident (latency-bound, not HBM-bound); host_io: lsg_batch_launch_io of the scan alone from "
                   "and to pinned host memory (x,y,z,r and elevations in; labels, count, mesh bytes and normals out), "
                   "events around each call, one call at a time")
    # the L2 side of the largest single scan, from the committed one-kernel
    # ncu capture of its tile kernel (null once the kernels have changed)
    vals = profiled_values("single_scan_k_tile.md")
    if vals:
        try:
            res["ring128x4096"]["k_tile_l2_frac"] = float(vals["lts_throughput_frac"])
            res["ring128x4096"]["k_tile_sm_frac"] = float(vals["sm_throughput_frac"])
            res["ring128x4096"]["k_tile_l2_bytes"] = float(vals["lts_bytes"])
            res["ring128x4096"]["l2_source"] = "profiles/single_scan_k_tile.md (ncu, lts__throughput and sm__throughput)"
        except (KeyError, ValueError):
            pass
    return res


def host_io_latency(ctx, scan, p, local, reps, warm):
    """End-to-end device time of one scan from and to pinned host memory:
    lsg_batch_launch_io with n = 1 (x,y,z,r and elevations in; labels, count,
    mesh bytes and normals out), events around each call, one call at a time
    as a request waits for its results; p50 / p99 of `reps` calls."""
    import torch

    from paper_2005_02704_gb300 import lsg
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    H, W, s_ = scan.rings, scan.cols, p.subsample
    Ws = lsg.ws_of(W, s_)
    hx = torch.empty(scan.xyzr.shape, dtype=torch.float32, pin_memory=True)
    hx.numpy()[...] = scan.xyzr
    he = torch.empty(H, dtype=torch.float32, pin_memory=True)
    he.numpy()[...] = scan.elev
    hl = torch.empty((H, W), dtype=torch.int32, pin_memory=True)
    hn = torch.empty(1, dtype=torch.int32, pin_memory=True)
    hm = torch.empty((H, Ws), dtype=torch.uint8, pin_memory=True)
    hv = torch.empty((H, Ws, 3), dtype=torch.float32, pin_memory=True)
    x = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    e = torch.empty(H, dtype=torch.float32, device=dev)
    out = lsg.alloc_outputs(H, W, s_, dev)
    io = (lsg.lsg_host_io * 1)()
    io[0].xyzr, io[0].elevation, io[0].labels = hx.data_ptr(), he.data_ptr(), hl.data_ptr()
    io[0].nseg, io[0].meshbits, io[0].normals = hn.data_ptr(), hm.data_ptr(), hv.data_ptr()
    sa = (lsg.lsg_scan * 1)(lsg.make_scan(e, xyzr=x, az0=scan.az0, daz=scan.daz))
    pa = (lsg.lsg_params * 1)(p.to_c())
    oa = (lsg.lsg_out * 1)(out.to_c())

    def call():
        rc = lsg.lsg_batch_launch_io(ctx.h, sa, pa, oa, io, stream.cuda_stream)
        if rc != lsg.LSG_OK:
            raise lsg.LsgError(rc, "lsg_batch_launch_io")

    for _ in range(warm):
        call()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    torch.cuda.synchronize()
    for a, b in ev:
        a.record(stream)
        call()
        b.record(stream)
        b.synchronize()
    if ctx.error() != lsg.LSG_OK:
        raise RuntimeError("device error in the host-buffer single-scan measurement")
    t = sorted(a.elapsed_time(b) for a, b in ev)
    return {"bytes_in": H * W * 16 + H * 4, "bytes_out": H * W * 4 + 4 + H * Ws * 13,
            "p50_ms": pct(t, 0.5), "p99_ms": pct(t, 0.99)}


def oracle_single_scans(reps=3):
    """The oracle's single-threaded time per single-scan workload (median of
    `reps` runs)."""
    import lidarsim
    import oracle as O
    res = {}
    for name, maker in SINGLE_SCANS:
        spec = getattr(lidarsim, maker)()
        scan = lidarsim.make_scan(spec)
        p = O.Params(subsample=spec.subsample, r_max=spec.r_max, jump_rel_h=spec.jump_rel_h,
                     jump_rel_v=spec.jump_rel_v, angle_rad=math.radians(spec.angle_deg))
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            O.segment_scan(scan, p)
            ts.append((time.perf_counter() - t0) * 1e3)
        ms = statistics.median(ts)
        res[name] = {"ms": ms, "points_per_s": scan.rings * scan.cols / (ms / 1e3)}
    return res


# The paper's own timings (Table 1: C++ on one 7th-generation i5 core, 32 x
# 1800 scans of 57,600 points), context only
PAPER_TABLE1 = {"hardware": "7th-generation Intel i5, DDR4 8 GB, C++ (thread count and precision not stated)",
                "scan": "32 x 1800 (57,600 points), simulated Velodyne 32E",
                "ms_per_scan": {"s=5": 54.33, "s=10": 35.06, "s=15": 25.53},
                "points_per_s": {"s=5": 57600 / 54.33e-3, "s=10": 57600 / 35.06e-3, "s=15": 57600 / 25.53e-3}}


def spin_measurement(local, tile, reps=20, packets=16):
    """Streaming: a 128 x 4096 scan (the 128-ring template, 0.088 deg) pushed
    in `packets` column ranges; device time from the last packet to labels
    ready (the finish, which takes the last packet's columns too) against
    one lsg_segment pass of the whole scan.  Medians over `reps`."""
    import torch

    import lidarsim
    from paper_2005_02704_gb300 import lsg
    dev = torch.device("cuda", local)
    spec = lidarsim.ring128()
    scan = lidarsim.make_scan(spec)
    p = lsg.Params(r_max=spec.r_max, jump_rel_h=spec.jump_rel_h, jump_rel_v=spec.jump_rel_v,
                   angle_rad=math.radians(spec.angle_deg))
    elev = torch.from_numpy(scan.elev).to(dev)
    xyzr = torch.from_numpy(scan.xyzr).to(dev)
    ctx = lsg.Context(local, tile=tile)
    out = lsg.alloc_outputs(scan.rings, scan.cols, 1, dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    full, last = [], []
    for k in range(reps + 3):
        torch.cuda.synchronize()
        e0.record()
        ctx.segment(elev, xyzr=xyzr, az0=scan.az0, daz=scan.daz, params=p, out=out)
        e1.record()
        torch.cuda.synchronize()
        if k >= 3:
            full.append(e0.elapsed_time(e1))
        spin = lsg.Spin(ctx, elev, xyzr=xyzr, az0=scan.az0, daz=scan.daz, params=p, out=out)
        for q in range(1, packets):
            spin.push(scan.cols * q // packets)
        torch.cuda.synchronize()
        e0.record()
        spin.finish()  # the last packet is in place: finish takes the rest
        e1.record()
        torch.cuda.synchronize()
        spin.close()
        if k >= 3:
            last.append(e0.elapsed_time(e1))
    ctx.close()
    f, l = statistics.median(full), statistics.median(last)
    tile_name = "auto (per call)" if tile == lsg.LSG_TILE_AUTO else next(k for k, v in lsg.TILES.items() if v == tile)
    return {"scan": f"{scan.rings}x{scan.cols} (128-ring template), {packets} packets", "tile": tile_name,
            "after_last_packet_ms": l, "full_pass_ms": f, "latency_cut": f / l}


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    from paper_2005_02704_gb300 import replicas
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if args.single_only:
        if rank == 0:
            print(json.dumps({"single_scans": single_scan_measurement(local, measured_hbm()[0],
                                                                     reps=args.steps, warm=args.warmup)}), flush=True)
        return
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    red = replicas.Reducer(world, device=torch.device("cuda", local))
    barrier, max_over_ranks, sum_over_ranks = red.barrier, red.max, red.sum

    from paper_2005_02704_gb300 import batch, lsg
    lsg.load()
    specs, scans = batch_data(args.scans, rank)
    shapes = [batch.ScanShape(s.rings, s.cols, sp.subsample) for sp, s in zip(specs, scans)]
    db = batch.DeviceBatch(shapes, [seg_params(sp) for sp in specs], local)
    for b, s in enumerate(scans):
        db.set_scan(b, s)
    db.upload()
    torch.cuda.synchronize()
    ctx = lsg.Context(local)
    plan = db.plan(ctx, lsg.TILES[args.tile] if args.tile else lsg.LSG_TILE_AUTO)
    stream = torch.cuda.current_stream()
    tuned = None
    if not args.no_autotune and not args.tile:
        tuned = plan.autotune(reps=3)
    if args.phased:
        plan.set_schedule(0)
    if args.fused:
        plan.set_schedule(1)
    if args.grouped:
        plan.set_schedule(2)
    schedule = plan.schedule
    launches_per_pass = plan.launches  # kernel launches in one replay (grouped: 1 + 3 per scan group)
    tile_name = {v: k for k, v in lsg.TILES.items()}[plan.tile]

    # ---- batched path, inputs resident ------------------------------------
    for _ in range(max(args.warmup, 3)):
        plan.run()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.run()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    ms_step = max_over_ranks(e0.elapsed_time(e1) / args.steps)
    if ctx.error() != lsg.LSG_OK:
        raise RuntimeError("device error during the timed region")
    pts_all = sum_over_ranks(float(db.points))
    value = pts_all / (ms_step / 1e3)
    # per-pass latency distribution: 100 single replays, events around each
    lat_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(100)]
    for a, b in lat_ev:
        a.record(stream)
        plan.run()
        b.record(stream)
    torch.cuda.synchronize()
    lat = sorted(a.elapsed_time(b) for a, b in lat_ev)
    batched_latency = {"p50_ms": pct(lat, 0.5), "p99_ms": pct(lat, 0.99), "passes": len(lat)}

    # ---- every schedule of the same plan and tile shape --------------------
    #      (K replays each, events on the launching stream)
    sched_ms = {}
    for sch, nm in (() if args.no_schedules else ((0, "phased"), (1, "fused"), (2, "grouped"))):
        plan.set_schedule(sch)
        for _ in range(3):
            plan.run()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            plan.run()
        e1.record(stream)
        torch.cuda.synchronize()
        sched_ms[nm] = max_over_ranks(e0.elapsed_time(e1) / args.steps)
    plan.set_schedule(schedule)
    if ctx.error() != lsg.LSG_OK:
        raise RuntimeError("device error while timing the schedules")

    # ---- per-phase device times (events recorded inside the graph) ---------
    # (the grouped schedule overlaps its kernels, so its per-kernel times are
    # taken from the phased capture of the same plan)
    phase = [0.0, 0.0, 0.0, 0.0]
    nrep = max(3, min(args.steps, 10))
    if schedule == 2:
        plan.set_schedule(0)
    for _ in range(nrep):
        plan.run()
        t = plan.phase_times()
        phase = [a + b for a, b in zip(phase, t)]
    phase = [x / nrep for x in phase]
    if schedule == 2:
        plan.set_schedule(2)

    # ---- end to end through the C ABI with host buffers --------------------
    # lsg_batch_plan_io: one graph replay per step copies every scan's inputs
    # from pinned host memory, runs the pass and copies every output (labels,
    # segment counts, mesh bytes, normals) back, in chunks whose copies in
    # both directions overlap the other chunks' passes; K replays between
    # events on the launching stream, median of three timed regions.  Also:
    # the same with one chunk (copies, pass and copies one after the other),
    # and the host link's floor for the same bytes (the input copy and the
    # output copy on two streams at once, nothing else).
    from paper_2005_02704_gb300 import serve

    def time_e2e(p_io):
        for _ in range(max(args.warmup, 3)):
            p_io.run(stream)
        regions = []
        with serve.no_gc_pauses():
            for _ in range(3):
                torch.cuda.synchronize()
                barrier()
                torch.cuda.synchronize()
                e0.record(stream)
                for _ in range(args.steps):
                    p_io.run(stream)
                e1.record(stream)
                torch.cuda.synchronize()
                barrier()
                regions.append(max_over_ranks(e0.elapsed_time(e1) / args.steps))
        if ctx.error() != lsg.LSG_OK:
            raise RuntimeError("device error in the end-to-end measurement")
        return statistics.median(regions), regions

    def link_floor(dbx):
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
        outs_h = (dbx.h_lab, dbx.h_nseg, dbx.h_mb, dbx.h_nrm)
        outs_d = (dbx.d_lab, dbx.d_nseg, dbx.d_mb, dbx.d_nrm)
        ts = []
        for k in range(4):
            torch.cuda.synchronize()
            e0.record(stream)
            s_in.wait_stream(stream)
            s_out.wait_stream(stream)
            with torch.cuda.stream(s_in):
                dbx.d_in.copy_(dbx.h_in, non_blocking=True)
                dbx.d_elev.copy_(dbx.h_elev, non_blocking=True)
            with torch.cuda.stream(s_out):
                for h, d_ in zip(outs_h, outs_d):
                    h.copy_(d_, non_blocking=True)
            stream.wait_stream(s_in)
            stream.wait_stream(s_out)
            e1.record(stream)
            torch.cuda.synchronize()
            if k:
                ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    e2e = None
    if not args.no_e2e:
        plan_io = db.plan_io(ctx, plan.tile, chunks=args.e2e_chunks)
        h2d, d2h = plan_io.io_bytes()
        ms_e2e, regions = time_e2e(plan_io)
        e2e_launches = plan_io.launches
        plan_io.close()
        plan_io1 = db.plan_io(ctx, plan.tile, chunks=1)
        ms_e2e_serial, _ = time_e2e(plan_io1)
        plan_io1.close()
        ms_floor = max_over_ranks(link_floor(db))
        e2e = {"value": pts_all / (ms_e2e / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e,
               "path": f"lsg_batch_plan_io + lsg_batch_run (C ABI) from pinned host buffers, "
                       f"{args.e2e_chunks} chunks in one graph: x,y,z,r and elevations in; labels, segment "
                       "counts, mesh bytes and normals out",
               "ms_per_step_regions": regions, "gpu_launches_per_step": e2e_launches,
               "serial_ms_per_step": ms_e2e_serial,
               "serial_value": pts_all / (ms_e2e_serial / 1e3),
               "serial_path": "the same plan with one chunk (copy in, pass, copy out in sequence)",
               "link_floor_ms": ms_floor,
               "link_floor_note": "the same bytes copied host->device and device->host on two streams at "
                                  "once, nothing else (torch copies of the pinned mirrors)"}
    # the device plan's outputs again (the host-buffer replays rewrote them)
    plan.run()
    torch.cuda.synchronize()

    # ---- the same batch as ranges only (the sensor's own output form) -------
    #     x,y,z decoded on the GPU from the ring elevation and column azimuth:
    #     a quarter of the input bytes, on the device and over the host link
    range_input = None
    if not args.no_range_input and not args.no_e2e:
        dbr = batch.DeviceBatch(shapes, [seg_params(sp) for sp in specs], local, form="range")
        for b, s_ in enumerate(scans):
            dbr.set_scan(b, s_)
        dbr.upload()
        planr = dbr.plan(ctx, plan.tile)
        planr.set_schedule(schedule)
        for _ in range(max(args.warmup, 3)):
            planr.run()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            planr.run()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms_r = max_over_ranks(e0.elapsed_time(e1) / args.steps)
        pior = dbr.plan_io(ctx, plan.tile, chunks=args.e2e_chunks)
        h2d_r, d2h_r = pior.io_bytes()
        ms_er, regions_r = time_e2e(pior)
        pior.close()
        planr.close()
        del dbr
        range_input = {"workload": "the same 512 scans, range float32 per point (x,y,z decoded on the GPU)",
                       "value": pts_all / (ms_r / 1e3), "unit": UNIT, "ms_per_step": ms_r,
                       "bytes_per_point": RANGE_PATH_BYTES_PER_POINT,
                       "e2e": {"value": pts_all / (ms_er / 1e3), "unit": UNIT, "ms_per_step": ms_er,
                               "ms_per_step_regions": regions_r, "h2d_bytes_per_step": h2d_r,
                               "d2h_bytes_per_step": d2h_r,
                               "path": f"lsg_batch_plan_io + lsg_batch_run (C ABI), {args.e2e_chunks} chunks; "
                                       "ranges and elevations in, labels, segment counts, mesh bytes and "
                                       "normals out"}}

    # ---- plain per-scan path: one lsg_segment call per scan ----------------
    plain = None
    if not args.no_plain:
        views = [(db.scan_inputs(b), db.view(b)) for b in range(db.n)]
        outs = [lsg.Outputs(*v) for _, v in views]
        prm = db.params

        def plain_pass():
            for b in range(db.n):
                (elev, xyzr), _ = views[b]
                ctx.segment(elev, xyzr=xyzr, az0=float(db.az0[b]), daz=float(db.daz[b]), params=prm[b],
                            out=outs[b], stream=stream)

        for _ in range(2):
            plain_pass()
        torch.cuda.synchronize()
        barrier()
        npl = max(2, min(args.steps, 5))
        from paper_2005_02704_gb300 import serve
        with serve.no_gc_pauses():
            e0.record(stream)
            t0 = time.perf_counter()
            for _ in range(npl):
                plain_pass()
            host_ms = (time.perf_counter() - t0) * 1e3 / npl  # enqueue time of the 512 calls
            e1.record(stream)
            torch.cuda.synchronize()
        ms_plain = max_over_ranks(e0.elapsed_time(e1) / npl)
        plain = {"value": pts_all / (ms_plain / 1e3), "unit": UNIT, "ms_per_pass": ms_plain,
                 "host_enqueue_ms_per_pass": host_ms,
                 "scans_per_s": db.n * world / (ms_plain / 1e3),
                 # a single-scan call of at most 256 rings launches three kernels (its
                 # tile kernel finds the ring order), a larger one four
                 "gpu_launches_per_pass": sum(3 if sh.rings <= 256 else 4 for sh in db.shapes),
                 "tile": "auto (per call)"}

    # ---- served path: continuous batching of 8 sensors vs a serial loop ---
    served = None
    spin = None
    if not args.no_spin and rank == 0:
        spin = spin_measurement(local, lsg.LSG_TILE_AUTO)
    singles = None
    if not args.no_single and rank == 0:
        singles = single_scan_measurement(local, measured_hbm()[0])
    generator = None
    if not args.no_generator:
        generator = generator_measurement(specs, local, max(3, min(args.steps, 5)), 2, max_over_ranks,
                                          sum_over_ranks)
    if not args.no_serve:
        served = serve_measurement(args, local, world, max_over_ranks, sum_over_ranks)
    accuracy = None
    if not args.no_accuracy and rank == 0:
        from paper_2005_02704_gb300 import evaluate
        rows = evaluate.table2(n_scenes=8)
        accuracy = {"protocol": "Sec. 3 edge-based precision / recall / F1, dilation radius 1, component predicate "
                                "I=J=K=0.2, 8 synthetic Velodyne-32E-like scenes (32 x 1800), ground truth = "
                                "primitive face per ray",
                    "rows": [{"interval": s_, "precision": p_, "recall": r_, "f1": f_} for s_, p_, r_, f_ in rows],
                    "paper_f1": {"5": 0.7406, "10": 0.7147, "15": 0.6910}}

    # ---- roofline of the dominant kernel ---------------------------------
    # the fused plan runs the whole pass in one persistent launch (k_fused),
    # whose algorithmic bytes are the path's; the phased plan's dominant
    # kernel is the tile kernel
    peak, peak_kind = measured_hbm()
    t_dom = phase[1] / 1e3
    fused = schedule == 1
    bpp = PATH_BYTES_PER_POINT if fused else TILE_BYTES_PER_POINT
    achieved = bpp * db.points / t_dom / 1e9
    traffic_pp = profiled_traffic("k_fused" if fused else "k_tile")
    roof = {"bound": "hbm",
            "kernel": ("k_fused (the whole pass in one persistent launch)" if fused else
                       "k_tile (decode+mesh+normals+edge mask+tile components)"),
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": f"{peak_kind} HBM copy bandwidth",
            "algorithmic_bytes_per_launch": bpp * db.points,
            "traffic": (traffic_pp * db.points) if traffic_pp is not None else None}
    path_achieved = PATH_BYTES_PER_POINT * db.points / (ms_step / 1e3) / 1e9

    # the path's roofline fraction of the other paths (the same 33 B/point)
    def path_frac(points_per_s):
        return PATH_BYTES_PER_POINT * points_per_s / 1e9 / peak

    if plain is not None:
        plain["path_roofline_frac"] = path_frac(plain["value"])
    if range_input is not None:
        range_input["path_roofline_frac"] = RANGE_PATH_BYTES_PER_POINT * range_input["value"] / 1e9 / peak
    if served is not None:
        for d in (served["batched"], served["serial_plain"], served["saturated"]["batched"],
                  served["saturated"]["serial_plain"]):
            d["path_roofline_frac"] = path_frac(d["points_per_s"])

    # ---- CPU baseline: the oracle on the host cores ------------------------
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cores = host_cores()
        r, pts, ns, dt = oracle_rate(specs, scans, float(db.points), cores)
        cpu = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{ns} of the 512 scans (every {math.ceil(len(scans) / ns)}th), {pts / 1e6:.1f} M points, "
                         f"{dt:.1f} s wall on {cores} threads",
               "single_scans_one_thread": oracle_single_scans() if not args.no_single else None}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(db.n, db.points, world),
            "plan": {"tile": tile_name, "schedule": SCHEDULES[schedule],
                     "autotune_ms": tuned[1] if tuned else None, "launches_per_pass": launches_per_pass},
            "schedule_ms": sched_ms,
            "roofline": roof,
            "path_roofline": {"bound": "hbm", "achieved": path_achieved, "peak": peak, "unit": "GB/s",
                              "frac": path_achieved / peak, "bytes_per_point": PATH_BYTES_PER_POINT,
                              # the aim on large batches: half of the HBM roofline
                              "target_frac": 0.5, "target_met": path_achieved / peak >= 0.5},
            "kernel_ms": ({"counter_reset": phase[0], "fused": phase[1]} if fused else
                          {"ring_order": phase[0], "tile": phase[1], "merge": phase[2], "labels": phase[3]}),
            "cpu_baseline": cpu,
            "e2e": e2e,
            "batched_latency": batched_latency,
            "range_input": range_input,
            "plain": plain,
            "single_scans": singles,
            "served": served,
            "generator": generator,
            "streaming": spin,
            "paper_table1": PAPER_TABLE1,
            "accuracy": accuracy,
            "scans_per_s": db.n * world / (ms_step / 1e3),
            "gpu_launches": launches_per_pass * args.steps,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

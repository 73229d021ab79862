"""Seeded synthetic spinning-Lidar scans (input generator).

The paper (Mukherjee et al., PReMI 2019, Sec. 3) simulates a Velodyne 32E
with Blensor over 32 primitive scenes (cylinders, spheres, cubes, cones on a
flat floor, Gaussian range noise).  That simulator needs a graphics stack and
its dataset is not public, so these scans stand in for it: a FP64 ray-caster
(``raycast.c``) over a ground plane (optionally sloped), axis-aligned boxes,
thin boxes used as walls and vertical cylinders, with Gaussian range noise,
random dropouts and a maximum range.

This module is shared by the tests, the oracle checks and the benchmark.  It
holds none of the segmentation arithmetic; it only draws scenes and casts
rays.  Scene placement uses a pure-Python SplitMix64 stream, so a scan is a
function of its seed on every machine.

Workload shapes (rings x columns, elevations, scene sizes, noise, dropouts)
follow the five benchmark workloads of this project:

* ``ring16``: 16 rings at -15..+15 deg (2 deg steps) x 1800 columns (0.2 deg),
  6 boxes and 4 cylinders within 40 m, sigma 1 cm, 5 % dropouts, 100 m.
* ``ring64``: 64 rings, theta_i = 2 - 26.8 (i/63)^1.5 deg, x 2048 columns,
  ground sloped up to 3 deg, 30 boxes, 20 cylinders, 2 walls within 120 m,
  sigma 2 cm, 3 % dropouts, sub-sampling 2, angle threshold 8 deg.
* ``ring128``: 128 rings at -25..+15 deg x 4096 columns, 100 boxes,
  60 cylinders, 4 walls within 150 m, sigma 2 cm, 2 % dropouts.
* ``batch512``: 512 scans, rings from {16, 32, 64, 128}, widths from
  {1024, 1800, 2048, 4096}; scene template chosen by the ring count.
* ``serve8``: 8 sensors with mixed ring counts for the serving simulation.
"""
from __future__ import annotations

import ctypes
import math
import os
import shutil
import subprocess
from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "raycast.c")
_LIB = os.path.join(_HERE, "liblidarsim.so")

M64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15

PRIM_PLANE, PRIM_BOX, PRIM_CYL = 0, 1, 2


# --------------------------------------------------------------------------
# build / load of the C ray-caster
# --------------------------------------------------------------------------
def build(force: bool = False) -> str:
    """Compile ``raycast.c`` into ``liblidarsim.so`` (OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler found for lidarsim")
    tmp = _LIB + f".tmp{os.getpid()}"
    base = [cc, "-O2", "-fPIC", "-shared", "-std=c99", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:2] + ["-fopenmp"] + base[2:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.lidarsim_raycast.restype = ctypes.c_int
        lib.lidarsim_raycast.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
            ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
            ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]
        _lib = lib
    return _lib


# --------------------------------------------------------------------------
# SplitMix64 scene-placement stream
# --------------------------------------------------------------------------
class SplitMix64:
    """SplitMix64 (Steele, Lea, Flood 2014): state += golden; mix(state)."""

    def __init__(self, seed: int):
        self.state = seed & M64

    def next_u64(self) -> int:
        self.state = (self.state + GOLDEN) & M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        return z ^ (z >> 31)

    def uniform(self, a: float = 0.0, b: float = 1.0) -> float:
        u = ((self.next_u64() >> 11) + 0.5) / 9007199254740992.0
        return a + (b - a) * u

    def randint(self, n: int) -> int:
        """Uniform integer in [0, n) by rejection (no modulo bias)."""
        lim = (1 << 64) - ((1 << 64) % n)
        while True:
            v = self.next_u64()
            if v < lim:
                return v % n

    def choice(self, seq):
        return seq[self.randint(len(seq))]


# --------------------------------------------------------------------------
# scene and sensor specification
# --------------------------------------------------------------------------
@dataclass
class SceneSpec:
    """One synthetic scan: sensor geometry, scene recipe, noise and the
    segmentation parameters the workload uses."""
    name: str
    elev_deg: List[float]            # ring elevations, in row order
    cols: int                        # W shots per revolution
    seed: int
    az0: float = 0.0
    ground_z: float = -1.7
    slope_max_deg: float = 0.0
    n_boxes: int = 0
    box_edge: tuple = (1.0, 5.0)
    n_cyl: int = 0
    cyl_rho: tuple = (0.1, 0.3)
    cyl_h: tuple = (1.0, 4.0)
    n_walls: int = 0
    wall_len: tuple = (20.0, 60.0)
    wall_h: tuple = (3.0, 8.0)
    wall_thick: float = 0.3
    scene_radius: float = 40.0
    min_dist: float = 3.0
    sigma: float = 0.01
    p_drop: float = 0.05
    r_max: float = 100.0
    # segmentation parameters for this workload
    subsample: int = 1
    angle_deg: float = 10.0
    jump_rel_h: float = 0.10
    jump_rel_v: float = 1.0
    extra_prims: list = field(default_factory=list)

    @property
    def rings(self) -> int:
        return len(self.elev_deg)

    @property
    def daz(self) -> float:
        return 2.0 * math.pi / self.cols


def elev_uniform(lo: float, hi: float, n: int) -> List[float]:
    if n == 1:
        return [lo]
    return [lo + (hi - lo) * i / (n - 1) for i in range(n)]


def elev_horizon_dense(n: int) -> List[float]:
    """theta_i = 2 - 26.8 (i/(n-1))^1.5 degrees, top ring first (denser near the horizon)."""
    return [2.0 - 26.8 * (i / (n - 1)) ** 1.5 for i in range(n)]


def ring16(seed: int = 1000, cols: int = 1800) -> SceneSpec:
    return SceneSpec("ring16", elev_uniform(-15.0, 15.0, 16), cols, seed,
                     n_boxes=6, n_cyl=4, scene_radius=40.0, sigma=0.01, p_drop=0.05,
                     r_max=100.0, subsample=1, angle_deg=10.0)


def ring64(seed: int = 1001, cols: int = 2048, rings: int = 64, subsample: int = 2,
           angle_deg: float = 8.0) -> SceneSpec:
    return SceneSpec("ring64", elev_horizon_dense(rings), cols, seed, slope_max_deg=3.0,
                     n_boxes=30, n_cyl=20, n_walls=2, scene_radius=120.0, sigma=0.02,
                     p_drop=0.03, r_max=120.0, subsample=subsample, angle_deg=angle_deg)


def ring128(seed: int = 1002, cols: int = 4096) -> SceneSpec:
    return SceneSpec("ring128", elev_uniform(-25.0, 15.0, 128), cols, seed,
                     n_boxes=100, n_cyl=60, n_walls=4, scene_radius=150.0, sigma=0.02,
                     p_drop=0.02, r_max=150.0, subsample=1, angle_deg=10.0)


BATCH_RINGS = (16, 32, 64, 128)
BATCH_COLS = (1024, 1800, 2048, 4096)


def batch_specs(n: int = 512, seed0: int = 2000) -> List[SceneSpec]:
    """The uneven batch: scan b has seed seed0+b, rings and width drawn from
    {16,32,64,128} x {1024,1800,2048,4096}; template by ring count
    (16 -> ring16, 32/64 -> ring64 law, 128 -> ring128); s=1, 10 deg."""
    specs = []
    for b in range(n):
        rng = SplitMix64(seed0 + b)
        h = rng.choice(BATCH_RINGS)
        w = rng.choice(BATCH_COLS)
        if h == 16:
            sp = ring16(seed0 + b, w)
        elif h in (32, 64):
            sp = ring64(seed0 + b, w, rings=h, subsample=1, angle_deg=10.0)
        else:
            sp = ring128(seed0 + b, w)
        specs.append(replace(sp, name=f"batch{b}"))
    return specs


def sensor_specs(n: int = 8, seed0: int = 3000) -> List[SceneSpec]:
    """Serving sensors: ring counts {16,32,64,128} two each, widths from the batch set."""
    specs = []
    for k in range(n):
        rng = SplitMix64(seed0 + k)
        h = BATCH_RINGS[k % 4]
        w = rng.choice(BATCH_COLS)
        if h == 16:
            sp = ring16(seed0 + k, w)
        elif h in (32, 64):
            sp = ring64(seed0 + k, w, rings=h, subsample=1, angle_deg=10.0)
        else:
            sp = ring128(seed0 + k, w)
        specs.append(replace(sp, name=f"sensor{k}"))
    return specs


# --------------------------------------------------------------------------
# scene placement
# --------------------------------------------------------------------------
def _rect_dist(x0, x1, y0, y1) -> float:
    dx = max(x0, 0.0, -x1)
    dy = max(y0, 0.0, -y1)
    return math.hypot(dx, dy)


def _ground(spec: SceneSpec, rng: SplitMix64):
    """Ground plane n.x = d through (0, 0, ground_z), tilted by up to slope_max_deg."""
    if spec.slope_max_deg > 0.0:
        tilt = math.radians(rng.uniform(-spec.slope_max_deg, spec.slope_max_deg))
        ax = rng.uniform(-math.pi, math.pi)  # horizontal rotation axis direction
        ux, uy = math.cos(ax), math.sin(ax)
        # rotate (0,0,1) about (ux,uy,0) by tilt: Rodrigues
        n = (uy * math.sin(tilt), -ux * math.sin(tilt), math.cos(tilt))
    else:
        n = (0.0, 0.0, 1.0)
    d = n[2] * spec.ground_z
    return n, d


def _ground_z(n, d, x, y) -> float:
    return (d - n[0] * x - n[1] * y) / n[2]


def scene_prims(spec: SceneSpec) -> np.ndarray:
    """Primitive table [n, 10] = kind, id, a[0..7] for the ray-caster."""
    rng = SplitMix64(spec.seed * 7919 + 17)
    prims = []
    n, d = _ground(spec, rng)
    prims.append([PRIM_PLANE, 0, n[0], n[1], n[2], d, 0, 0, 0, 0])
    pid = 1
    R = spec.scene_radius

    def place(half_x, half_y):
        for _ in range(1000):
            r = rng.uniform(spec.min_dist, R)
            a = rng.uniform(-math.pi, math.pi)
            cx, cy = r * math.cos(a), r * math.sin(a)
            if _rect_dist(cx - half_x, cx + half_x, cy - half_y, cy + half_y) >= spec.min_dist:
                return cx, cy
        raise RuntimeError("scene placement failed")

    for _ in range(spec.n_boxes):
        ex, ey, ez = (rng.uniform(*spec.box_edge) for _ in range(3))
        cx, cy = place(ex / 2, ey / 2)
        zg = _ground_z(n, d, cx, cy) - 0.25
        prims.append([PRIM_BOX, pid, cx - ex / 2, cy - ey / 2, zg, cx + ex / 2, cy + ey / 2, zg + ez, 0, 0])
        pid += 1
    for _ in range(spec.n_walls):
        ln = rng.uniform(*spec.wall_len)
        ht = rng.uniform(*spec.wall_h)
        along_x = rng.uniform() < 0.5
        hx, hy = (ln / 2, spec.wall_thick / 2) if along_x else (spec.wall_thick / 2, ln / 2)
        cx, cy = place(hx, hy)
        zg = _ground_z(n, d, cx, cy) - 0.5
        prims.append([PRIM_BOX, pid, cx - hx, cy - hy, zg, cx + hx, cy + hy, zg + ht, 0, 0])
        pid += 1
    for _ in range(spec.n_cyl):
        rho = rng.uniform(*spec.cyl_rho)
        h = rng.uniform(*spec.cyl_h)
        cx, cy = place(rho, rho)
        zg = _ground_z(n, d, cx, cy) - 0.25
        prims.append([PRIM_CYL, pid, cx, cy, rho, zg, zg + h, 0, 0, 0])
        pid += 1
    for p in spec.extra_prims:
        q = list(p) + [0] * (10 - len(p))
        q[1] = pid
        prims.append(q[:10])
        pid += 1
    return np.ascontiguousarray(np.array(prims, dtype=np.float64))


@dataclass
class Scan:
    """A ray-cast scan.  Rows are in the order of ``elev`` (not sorted)."""
    spec: SceneSpec
    xyzr: np.ndarray       # float32 [H, W, 4]
    gt: np.ndarray         # int32 [H, W]: prim id * 8 + face, -1 = no return
    elev: np.ndarray       # float32 [H] radians
    az0: float             # float32-representable
    daz: float

    @property
    def range(self) -> np.ndarray:
        return np.ascontiguousarray(self.xyzr[..., 3])

    @property
    def rings(self) -> int:
        return self.xyzr.shape[0]

    @property
    def cols(self) -> int:
        return self.xyzr.shape[1]

    @property
    def points(self) -> int:
        return self.rings * self.cols


def raycast(spec: SceneSpec, prims: Optional[np.ndarray] = None, sigma: Optional[float] = None,
            p_drop: Optional[float] = None) -> Scan:
    """Cast every ray of ``spec`` against ``prims`` (default: the spec's scene)."""
    lib = _load()
    if prims is None:
        prims = scene_prims(spec)
    prims = np.ascontiguousarray(prims, dtype=np.float64)
    H, W = spec.rings, spec.cols
    elev32 = np.array([math.radians(e) for e in spec.elev_deg], dtype=np.float32)
    az0 = float(np.float32(spec.az0))
    daz = float(np.float32(spec.daz))
    elev64 = elev32.astype(np.float64)
    xyzr = np.zeros((H, W, 4), dtype=np.float32)
    gt = np.full((H, W), -1, dtype=np.int32)
    rc = lib.lidarsim_raycast(H, W, elev64.ctypes.data, az0, daz, prims.shape[0], prims.ctypes.data,
                              spec.sigma if sigma is None else sigma,
                              spec.p_drop if p_drop is None else p_drop,
                              spec.r_max, spec.seed & M64, xyzr.ctypes.data, gt.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"lidarsim_raycast failed: {rc}")
    return Scan(spec, xyzr, gt, elev32, az0, daz)


def make_scan(spec: SceneSpec) -> Scan:
    return raycast(spec)

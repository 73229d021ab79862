"""CPU checks of the scan generators: the CPU FP64 ray-caster against closed
forms and its noise model against its stated distribution (it is the
reference the GPU generator is compared with), and host-side argument
validation of lsg_raycast (no device needed)."""
import ctypes
import math

import numpy as np

import lidarsim
from paper_2005_02704_gb300 import lsg


def plane_scene(n, d):
    return np.array([[lidarsim.PRIM_PLANE, 0, n[0], n[1], n[2], d, 0, 0, 0, 0]], dtype=np.float64)


def directions(scan):
    el = scan.elev.astype(np.float64)[:, None]
    ph = scan.az0 + np.arange(scan.cols, dtype=np.float64)[None, :] * scan.daz
    return np.stack([np.cos(el) * np.cos(ph), np.cos(el) * np.sin(ph), np.sin(el) + 0 * ph], -1)


def test_cpu_ground_plane_closed_form():
    """Noiseless tilted plane n.p = d: every downward ray returns d / (n.dir)
    (to float32 rounding of r), every upward ray nothing."""
    spec = lidarsim.SceneSpec("g", lidarsim.elev_uniform(-20.0, 10.0, 13), 720, seed=5, sigma=0.0, p_drop=0.0,
                              r_max=200.0)
    n = np.array([0.03, -0.02, 1.0])
    n /= np.linalg.norm(n)
    scan = lidarsim.raycast(spec, prims=plane_scene(n, -1.7))
    dirs = directions(scan)
    nd = dirs @ n
    t = -1.7 / nd
    hit = (nd < 0) & (t <= 200.0)
    r = scan.xyzr[..., 3].astype(np.float64)
    assert np.all((r > 0) == hit)
    assert np.all(np.abs(r[hit] - t[hit]) <= 2.0 ** -23 * t[hit])
    assert np.all(scan.gt[hit] == 0) and np.all(scan.gt[~hit] == -1)
    # the point lies on the plane up to float32 rounding of x, y, z
    p = scan.xyzr[..., :3].astype(np.float64)
    assert np.all(np.abs(p[hit] @ n + 1.7) <= 4 * 2.0 ** -24 * (np.abs(p[hit]).sum(-1) + 1.7))


def test_cpu_cylinder_and_box_faces():
    """Horizontal rays toward a cylinder's axis return dist - rho on face 0;
    the ray along +x into a box enters its min-x face (face 0)."""
    spec = lidarsim.SceneSpec("c", [0.0], 360, seed=1, sigma=0.0, p_drop=0.0, r_max=100.0)
    prims = np.array([[lidarsim.PRIM_CYL, 3, 10.0, 0.0, 0.5, -1.0, 1.0, 0, 0, 0],
                      [lidarsim.PRIM_BOX, 4, -8.0, -1.0, -1.0, -6.0, 1.0, 1.0, 0, 0]], dtype=np.float64)
    scan = lidarsim.raycast(spec, prims=prims)
    c0 = int(round((0.0 - scan.az0) / scan.daz)) % scan.cols
    assert scan.gt[0, c0] == 3 * 8 + 0
    assert abs(scan.xyzr[0, c0, 3] - 9.5) <= 1e-5
    c180 = int(round((math.pi - scan.az0) / scan.daz)) % scan.cols
    assert scan.gt[0, c180] == 4 * 8 + 1  # the max-x face (x = -6) faces the sensor
    assert abs(scan.xyzr[0, c180, 3] - 6.0) <= 1e-5


def test_cpu_noise_and_dropout_statistics():
    """Range noise is N(0, sigma) and dropouts Bernoulli(p): the sample mean,
    variance and dropout fraction stay within 5 standard errors."""
    sigma, p = 0.05, 0.1
    spec = lidarsim.SceneSpec("n", lidarsim.elev_uniform(-30.0, -10.0, 16), 2048, seed=11, sigma=sigma, p_drop=p,
                              r_max=200.0)
    prims = plane_scene(np.array([0.0, 0.0, 1.0]), -2.0)
    noisy = lidarsim.raycast(spec, prims=prims)
    clean = lidarsim.raycast(spec, prims=prims, sigma=0.0, p_drop=0.0)
    r, t = noisy.xyzr[..., 3].astype(np.float64), clean.xyzr[..., 3].astype(np.float64)
    kept = r > 0
    n = t.size
    frac = 1.0 - kept.mean()
    assert abs(frac - p) <= 5 * math.sqrt(p * (1 - p) / n)
    e = (r - t)[kept]
    m = e.size
    assert abs(e.mean()) <= 5 * sigma / math.sqrt(m)
    assert abs(e.var() / sigma ** 2 - 1.0) <= 5 * math.sqrt(2.0 / m)


def test_raycast_spec_layout():
    assert ctypes.sizeof(lsg.lsg_raycast_spec) == 72
    assert lsg.lsg_raycast_spec.prims.offset == 32
    assert lsg.lsg_raycast_spec.seed.offset == 64


def test_raycast_rejects_bad_arguments_without_a_device():
    lib = lsg.load()
    assert lib.lsg_raycast(None, None, None, None) == lsg.LSG_E_ARG
    s = lsg.lsg_raycast_spec()
    s.rings, s.cols, s.nprims, s.sigma, s.p_drop, s.r_max = 4, 8, 0, 0.0, 0.0, 10.0
    assert lsg.lsg_raycast(s, 0, 0) == lsg.LSG_E_ARG                      # no output buffer
    s.nprims = lsg.LSG_RAYCAST_MAX_PRIMS + 1
    assert lsg.lsg_raycast(s, 16, 0) == lsg.LSG_E_ARG                     # too many primitives
    s.nprims, s.p_drop = 0, 1.5
    assert lsg.lsg_raycast(s, 16, 0) == lsg.LSG_E_ARG                     # probability out of range
    s.p_drop, s.rings, s.cols = 0.0, 1 << 16, 1 << 16
    assert lsg.lsg_raycast(s, 16, 0) == lsg.LSG_E_SHAPE                   # more than LSG_MAX_POINTS
    s.rings, s.cols = 4, 8
    assert lsg.lsg_raycast(s, 8, 0) == lsg.LSG_E_ARG                      # xyzr not 16-byte aligned
    s.rings = 0
    assert lsg.lsg_raycast(s, 16, 0) == lsg.LSG_OK                        # empty: nothing launched

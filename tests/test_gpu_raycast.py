"""GPU scan generator (lsg_raycast) against the CPU FP64 ray-caster on the
same scenes, rays, seeds and counter-based random draws.

Bar: the surface hit (ground-truth id, which includes every dropout and
range-cut decision) agrees on all but a few grazing / edge rays; where both
return a point, the range agrees to the float32 evaluation of the
intersection, |dr| <= 8 u_32 t / cos + 1e-5 m, with cos the ray's angle of
incidence against the surface (the float32 ray parameter of a plane or slab
hit is a quotient of a dot product that loses relative accuracy as the ray
grazes), and x, y, z agree to the same bound."""
import math

import numpy as np
import pytest

import lidarsim

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U32 = 2.0 ** -24


def gpu_scan(spec, prims=None, sigma=None, p_drop=None):
    from paper_2005_02704_gb300 import lsg
    dev = torch.device("cuda", 0)
    prims = lidarsim.scene_prims(spec) if prims is None else prims
    elev = torch.tensor([math.radians(e) for e in spec.elev_deg], dtype=torch.float32, device=dev)
    xyzr, gt = lsg.raycast(elev, spec.cols, float(np.float32(spec.az0)), float(np.float32(spec.daz)),
                           torch.from_numpy(np.ascontiguousarray(prims, dtype=np.float64)).to(dev),
                           spec.sigma if sigma is None else sigma, spec.p_drop if p_drop is None else p_drop,
                           spec.r_max, spec.seed)
    torch.cuda.synchronize()
    return xyzr.cpu().numpy(), gt.cpu().numpy()


def incidence_cos(scan, prims):
    """|cos| of the angle between each CPU ray and the normal of the face it
    hit (1 where nothing was hit)."""
    el = scan.elev.astype(np.float64)[:, None]
    ph = scan.az0 + np.arange(scan.cols, dtype=np.float64)[None, :] * scan.daz
    d = np.stack([np.cos(el) * np.cos(ph), np.cos(el) * np.sin(ph), np.sin(el) + 0 * ph], -1)
    row_of = np.zeros(int(prims[:, 1].max()) + 1, np.int64)
    row_of[prims[:, 1].astype(np.int64)] = np.arange(len(prims))
    g = scan.gt
    hit = g >= 0
    pr = prims[row_of[np.where(hit, g // 8, 0)]]
    face = g % 8
    kind = pr[..., 0].astype(np.int64)
    p = scan.xyzr[..., :3].astype(np.float64)
    n = np.zeros(g.shape + (3,))
    plane = kind == lidarsim.PRIM_PLANE
    n[plane] = pr[plane][:, 2:5]
    box = kind == lidarsim.PRIM_BOX
    n[box, face[box] // 2] = 1.0
    side = (kind == lidarsim.PRIM_CYL) & (face == 0)
    n[side, 0] = p[side, 0] - pr[side][:, 2]
    n[side, 1] = p[side, 1] - pr[side][:, 3]
    cap = (kind == lidarsim.PRIM_CYL) & (face != 0)
    n[cap, 2] = 1.0
    cosi = np.abs((d * n).sum(-1)) / np.maximum(np.linalg.norm(n, axis=-1), 1e-300)
    return np.where(hit, cosi, 1.0)


SPECS = [lidarsim.ring16(), lidarsim.ring64(), lidarsim.ring128(cols=1024)] + lidarsim.batch_specs(6, seed0=8100)


@pytest.mark.parametrize("spec", SPECS, ids=[f"{s.name}-{s.rings}x{s.cols}-{s.seed}" for s in SPECS])
def test_gpu_generator_matches_cpu(gpu_lib, spec):
    cpu = lidarsim.make_scan(spec)
    prims = lidarsim.scene_prims(spec)
    xyzr, gt = gpu_scan(spec, prims)
    n = gt.size
    same = gt == cpu.gt
    # different surfaces only on rays that graze an edge or a silhouette
    assert (~same).sum() <= max(3, 2e-4 * n), f"{(~same).sum()} of {n} rays hit a different surface"
    both = same & (cpu.gt >= 0)
    r_c = cpu.xyzr[..., 3].astype(np.float64)
    r_g = xyzr[..., 3].astype(np.float64)
    cosi = incidence_cos(cpu, prims)
    tol = 8 * U32 * r_c / np.maximum(cosi, 1e-3) + 1e-5
    err = np.abs(r_g - r_c)
    assert np.all(err[both] <= tol[both]), f"max range error {err[both].max():.3g}"
    exyz = np.abs(xyzr[..., :3].astype(np.float64) - cpu.xyzr[..., :3]).max(-1)
    assert np.all(exyz[both] <= tol[both] + 2 * U32 * r_c[both])
    assert np.all(xyzr[~(gt >= 0)] == 0.0)
    print(f"\n{spec.name}: {(~same).sum()} of {n} rays differ; max |dr| {err[both].max():.3g} m")


def test_gpu_generator_ground_plane_closed_form(gpu_lib):
    spec = lidarsim.SceneSpec("g", lidarsim.elev_uniform(-20.0, 10.0, 13), 720, seed=5, sigma=0.0, p_drop=0.0,
                              r_max=200.0)
    nrm = np.array([0.03, -0.02, 1.0])
    nrm /= np.linalg.norm(nrm)
    prims = np.array([[lidarsim.PRIM_PLANE, 0, *nrm, -1.7, 0, 0, 0, 0]])
    xyzr, gt = gpu_scan(spec, prims)
    el = np.radians(np.array(spec.elev_deg, dtype=np.float32).astype(np.float64))[:, None]
    az0, daz = float(np.float32(spec.az0)), float(np.float32(spec.daz))
    ph = az0 + np.arange(spec.cols)[None, :] * daz
    d = np.stack([np.cos(el) * np.cos(ph), np.cos(el) * np.sin(ph), np.sin(el) + 0 * ph], -1)
    nd = d @ nrm
    t = -1.7 / nd
    hit = (nd < 0) & (t <= 200.0)
    assert np.all((gt >= 0) == hit)
    cosi = np.abs(nd)
    assert np.all(np.abs(xyzr[..., 3][hit] - t[hit]) <= 8 * U32 * t[hit] / cosi[hit] + 1e-6)


def test_gpu_generator_edge_cases(gpu_lib):
    from paper_2005_02704_gb300 import lsg
    dev = torch.device("cuda", 0)
    elev = torch.zeros(3, dtype=torch.float32, device=dev)
    empty = torch.zeros((0, 10), dtype=torch.float64, device=dev)
    xyzr, gt = lsg.raycast(elev, 5, 0.0, 0.1, empty, 0.01, 0.0, 50.0, 1)
    torch.cuda.synchronize()
    assert torch.all(gt == -1) and torch.all(xyzr == 0)
    # p_drop = 1 removes every return
    spec = lidarsim.ring16(cols=256)
    xyzr, gt = gpu_scan(spec, p_drop=1.0)
    assert np.all(gt == -1) and np.all(xyzr == 0.0)

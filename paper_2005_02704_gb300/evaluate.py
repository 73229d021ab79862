"""Edge-based segmentation accuracy (the paper's protocol, Sec. 3).

Segments carry no semantic labels, so the paper compares segment boundaries:
the boundary points of the segmentation and of the ground truth are each
dilated, and precision / recall count the boundary points of one that fall
on the dilated boundary of the other.  Here the ground truth is the face id
of the surface each ray hit in the synthetic scene (``lidarsim``), which
stands in for the Blensor annotations of the paper's dataset.

Boundary point: a point (in range) whose label differs from that of a
neighbouring point in range on its ring (previous / next shot, wrapping) or
in the same column on the adjacent rings.  Dilation: a (2r+1) x (2r+1)
window on the ring-by-shot grid (shots wrap).

Run ``python -m paper_2005_02704_gb300.evaluate`` on a GPU to print the
accuracy of the CUDA path at sub-sampling 5, 10 and 15 on synthetic
Velodyne-32E-like scans (32 rings x 1800 shots, 0.2 deg; primitives on a
flat floor), the setting of the paper's Table 2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def boundary(ids: np.ndarray, valid: np.ndarray) -> np.ndarray:
    """Points in range whose id differs from a neighbour in range (4-neighbourhood,
    shots wrap around the spin)."""
    H, W = ids.shape
    out = np.zeros((H, W), bool)
    for di, dj in ((0, 1), (0, -1), (1, 0), (-1, 0)):
        nb = np.roll(ids, shift=(-di, -dj), axis=(0, 1))
        nv = np.roll(valid, shift=(-di, -dj), axis=(0, 1))
        if di == 1:
            nv[-1, :] = False
        if di == -1:
            nv[0, :] = False
        out |= valid & nv & (nb != ids)
    return out


def dilate(mask: np.ndarray, r: int) -> np.ndarray:
    """Square dilation of radius r on the ring-by-shot grid (shots wrap)."""
    H, _ = mask.shape
    out = mask.copy()
    for di in range(-r, r + 1):
        for dj in range(-r, r + 1):
            if di == 0 and dj == 0:
                continue
            sh = np.roll(mask, shift=dj, axis=1)
            if di > 0:
                sh = np.vstack([np.zeros((di, mask.shape[1]), bool), sh[:H - di]])
            elif di < 0:
                sh = np.vstack([sh[-di:], np.zeros((-di, mask.shape[1]), bool)])
            out |= sh
    return out


@dataclass
class PRF:
    precision: float
    recall: float
    f1: float
    n_pred: int
    n_gt: int


def edge_prf(labels: np.ndarray, gt: np.ndarray, radius: int = 1) -> PRF:
    """Precision / recall / F1 of the segmentation's boundary points against the
    ground truth's, with dilation radius `radius`.  labels, gt: [H, W] in the
    same ring order; points with gt < 0 (no return) and labels < 0 are not
    points of either boundary."""
    valid = (gt >= 0) & (labels >= 0)
    pb = boundary(labels, valid)
    gb = boundary(gt, valid)
    n_p, n_g = int(pb.sum()), int(gb.sum())
    prec = float((pb & dilate(gb, radius)).sum() / n_p) if n_p else 1.0
    rec = float((gb & dilate(pb, radius)).sum() / n_g) if n_g else 1.0
    f1 = 2 * prec * rec / (prec + rec) if prec + rec > 0 else 0.0
    return PRF(prec, rec, f1, n_p, n_g)


def velodyne32_scene(seed: int):
    """A Velodyne-32E-like scan spec (32 rings from -30.67 to +10.67 deg,
    1800 shots, 0.2 deg) over primitives on a flat floor."""
    import lidarsim
    elev = [-30.67 + 1.333 * i for i in range(32)]
    return lidarsim.SceneSpec("velodyne32", elev, 1800, seed, n_boxes=8, n_cyl=6, scene_radius=25.0, sigma=0.01,
                              p_drop=0.0, r_max=80.0, jump_rel_v=1.0)


def table2(n_scenes: int = 8, intervals=(5, 10, 15), radius: int = 1, predicate: str = "component"):
    """Mean precision / recall / F1 of the CUDA path over synthetic scenes for
    each sampling interval (paper's thresholds I = J = K = 0.2 by default)."""
    import torch

    import lidarsim
    from . import lsg
    dev = torch.device("cuda", 0)
    ctx = lsg.Context(0)
    rows = []
    for s in intervals:
        acc = []
        for k in range(n_scenes):
            spec = velodyne32_scene(4000 + k)
            scan = lidarsim.make_scan(spec)
            p = lsg.Params(subsample=s, r_max=spec.r_max, jump_rel_h=spec.jump_rel_h, jump_rel_v=spec.jump_rel_v,
                           predicate=lsg.LSG_PRED_COMPONENT if predicate == "component" else lsg.LSG_PRED_ANGLE,
                           angle_rad=math.radians(10.0), comp=(0.2, 0.2, 0.2))
            out = ctx.segment(torch.from_numpy(scan.elev).to(dev), xyzr=torch.from_numpy(scan.xyzr).to(dev),
                              az0=scan.az0, daz=scan.daz, params=p)
            order = np.lexsort((np.arange(scan.rings), -scan.elev.astype(np.float64)))
            acc.append(edge_prf(out.labels.cpu().numpy(), scan.gt[order], radius))
        rows.append((s, float(np.mean([a.precision for a in acc])), float(np.mean([a.recall for a in acc])),
                     float(np.mean([a.f1 for a in acc]))))
    ctx.close()
    return rows


if __name__ == "__main__":
    print("interval  precision  recall  F1")
    for s, p, r, f in table2():
        print(f"{s:8d}  {p:9.4f}  {r:6.4f}  {f:.4f}")

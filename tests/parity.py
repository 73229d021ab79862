"""Comparison of the CUDA path with the FP64 oracle (shared by the GPU tests
and the smoke check).

Tolerances are derived from the binary32 arithmetic of the kernels:

* mesh bits and validity: bit-exact (the cut is decided in binary32 on both
  sides, validity is a float comparison);
* normals: the kernel's spoke differences, cross products, weights and sums
  each add at most a few units of u = 2^-24 relative to sum_k w_k |V_k||V_k+1|,
  so the angle error is at most  B = 36 u kappa + 6 u  with
  kappa = sum_k w_k |V_k||V_k+1| / |sum_k w_k V_k x V_k+1|  (factor 2 of
  safety over the term count).  In range-only decode the binary32 x,y,z carry
  an extra error e <= 2 r u (|phi|max + 8) per point, which moves the normal by
  at most 4 e ntri / |sum| (since sum_k w_k (|V_k| + |V_k+1|) = ntri).
  Vertices with B <= 1e-4 must meet the 1e-4 rad bar; the others (reported as
  ill-conditioned) must meet their own B;
* edge mask: equal outside a band |margin| <= B_p + B_q + 12 u / sin(theta_t)
  (angle form) or B_p + B_q + 4 u (component form); edges in the band are
  counted;
* labels: bit-exact given the same edge mask, both ways.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

import oracle as O

U = 2.0 ** -24
NORMAL_TOL = 1e-4
BIT_MESH = O.BIT_R | O.BIT_D | O.BIT_G


def oracle_params(p) -> O.Params:
    return O.Params(subsample=p.subsample, r_min=p.r_min, r_max=p.r_max, jump_rel_h=p.jump_rel_h,
                    jump_rel_v=p.jump_rel_v, predicate=p.predicate, angle_rad=p.angle_rad,
                    comp=tuple(p.comp), wrap=p.wrap)


def normal_bounds(orc: O.Result, range_only: bool = False, ranges=None, phi_max: float = 0.0,
                  s: int = 1) -> np.ndarray:
    with np.errstate(invalid="ignore", over="ignore", divide="ignore"):
        b = 36.0 * U * orc.kappa + 6.0 * U
        if range_only:
            r_v = ranges[:, ::s].astype(np.float64)
            e = 2.0 * r_v * U * (abs(phi_max) + 8.0)
            b = b + 4.0 * e * orc.ntri / orc.snorm
    b = np.where(np.isfinite(b), b, np.inf)
    return b


def angle_between(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    cr = np.cross(a, b)
    return np.arctan2(np.linalg.norm(cr, axis=-1), np.sum(a * b, axis=-1))


@dataclass
class Report:
    vertices: int = 0
    ill_conditioned: int = 0
    max_err_well: float = 0.0
    max_err_all: float = 0.0
    frac_within_tol: float = 1.0
    edges: int = 0
    in_band: int = 0
    hasn_mismatch: int = 0
    edge_mismatch_outside_band: int = 0
    notes: list = field(default_factory=list)


def neighbour_index(H, Ws, wrap_eff):
    """Flat index of the R, D, G neighbour of every vertex (or -1)."""
    i, j = np.meshgrid(np.arange(H), np.arange(Ws), indexing="ij")
    jn = j + 1
    has_r = (jn < Ws) | bool(wrap_eff)
    jn = np.where(jn >= Ws, 0, jn)
    r = np.where(has_r, i * Ws + jn, -1)
    d = np.where(i + 1 < H, (i + 1) * Ws + j, -1)
    g = np.where((i + 1 < H) & has_r, (i + 1) * Ws + jn, -1)
    return np.stack([r, d, g], axis=-1)


def compare_geometry(mb_g, nrm_g, orc: O.Result, p, bounds: np.ndarray, strict=True) -> Report:
    """Checks mesh bits, normals and the edge mask of one scan."""
    rep = Report()
    mb_o = orc.meshbits
    H, Ws = mb_o.shape
    rep.vertices = int(((mb_o & O.BIT_VALID) > 0).sum())
    keep = BIT_MESH | O.BIT_VALID
    if not np.array_equal(mb_g & keep, mb_o & keep):
        bad = np.argwhere((mb_g & keep) != (mb_o & keep))
        raise AssertionError(f"mesh bits differ at {len(bad)} vertices, first {bad[:5].tolist()}")
    has_o = (mb_o & O.BIT_HASN) > 0
    has_g = (mb_g & O.BIT_HASN) > 0
    mism = has_o != has_g
    rep.hasn_mismatch = int(mism.sum())
    hopeless = bounds >= math.pi / 2
    if strict:
        assert not (mism & ~hopeless).any(), "has-normal flag differs on a conditioned vertex"
    both = has_o & has_g
    err = np.zeros((H, Ws))
    if both.any():
        err[both] = angle_between(nrm_g[both].astype(np.float64), orc.normals[both])
    well = both & (bounds <= NORMAL_TOL)
    rep.ill_conditioned = int((both & ~well).sum())
    rep.max_err_well = float(err[well].max()) if well.any() else 0.0
    rep.max_err_all = float(err[both].max()) if both.any() else 0.0
    rep.frac_within_tol = float((err[both] <= NORMAL_TOL).mean()) if both.any() else 1.0
    if strict:
        assert rep.max_err_well <= NORMAL_TOL, f"normal error {rep.max_err_well} rad on a well-conditioned vertex"
        over = both & ~well & (err > bounds)
        assert not over.any(), f"{int(over.sum())} ill-conditioned normals exceed their bound"
    # edge mask
    nb = neighbour_index(H, Ws, p.wrap and Ws >= 3)
    ebits = (O.BIT_R, O.BIT_D, O.BIT_G)
    hbits = (O.BIT_HR, O.BIT_HD, O.BIT_HG)
    Bflat = np.minimum(bounds, math.pi).ravel()
    hasn_bad = mism.ravel()
    mbo = mb_o.ravel()
    mbg = mb_g.ravel()
    if p.predicate == O.PRED_ANGLE:
        extra = 12.0 * U / max(math.sin(p.angle_rad), 1e-3)
    else:
        extra = 4.0 * U
    for e in range(3):
        exists = (mbo & ebits[e]) > 0
        idx = np.nonzero(exists)[0]
        q = nb.reshape(-1, 3)[idx, e]
        rep.edges += len(idx)
        margin = orc.margin.reshape(-1, 3)[idx, e]
        delta = Bflat[idx] + Bflat[q] + extra
        band = np.isfinite(margin) & (np.abs(margin) <= delta)
        skip = band | hasn_bad[idx] | hasn_bad[q]
        rep.in_band += int(band.sum())
        go = (mbg[idx] & hbits[e]) > 0
        oo = (mbo[idx] & hbits[e]) > 0
        bad = (go != oo) & ~skip
        rep.edge_mismatch_outside_band += int(bad.sum())
    if strict:
        assert rep.edge_mismatch_outside_band == 0, f"{rep.edge_mismatch_outside_band} edge predicates differ outside the band"
    return rep


def sorted_valid(scan, p, order) -> np.ndarray:
    rs = scan.range[order]
    return ((np.float32(p.r_min) < rs) & (rs <= np.float32(p.r_max))).astype(np.uint8)


def check_outputs(ctx, scan, p, mb, nrm, lab, nseg, range_only=False, strict=True) -> Report:
    """The CUDA path's outputs of one scan (numpy: mesh bytes, normals, labels,
    segment count) against the oracle on the same scan: geometry within the
    bars above; labels and segment count exact under the same mask both ways
    (the oracle's components of the GPU mask, and ``ctx.label_from_mask`` of
    the oracle's mask, a GPU call); everything equal when the masks agree."""
    import torch
    orc = O.segment_scan(scan, oracle_params(p), range_only=range_only)
    phi_max = abs(scan.az0) + scan.cols * abs(scan.daz)
    bounds = normal_bounds(orc, range_only, scan.range[orc.order], phi_max, p.subsample)
    rep = compare_geometry(mb, nrm, orc, oracle_params(p), bounds, strict=strict)
    valid = sorted_valid(scan, p, orc.order)
    W, s, wrap = scan.cols, p.subsample, p.wrap
    lab_o_from_g, n_o_from_g = O.label_from_mask(mb, valid, W, s, wrap)
    assert np.array_equal(lab, lab_o_from_g)
    assert nseg == n_o_from_g
    dev = torch.device("cuda", 0)
    lab_g_from_o, n_g = ctx.label_from_mask(torch.from_numpy(orc.meshbits).to(dev),
                                            torch.from_numpy(valid).to(dev), W, s, wrap)
    torch.cuda.synchronize()
    assert np.array_equal(lab_g_from_o.cpu().numpy(), orc.labels)
    assert int(n_g.cpu()[0]) == orc.nseg
    if np.array_equal(mb, orc.meshbits):
        assert np.array_equal(lab, orc.labels) and nseg == orc.nseg
    return rep

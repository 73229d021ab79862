"""Pins of the FP64 oracle against things other than itself.

Each test checks one step of the path (Mukherjee et al., PReMI 2019, Sec. 2
and Algorithm 1) against a closed form, a brute-force enumeration on tiny
inputs, a hand-worked fixture, the paper's literal Algorithm 1, or an
invariant that a plausible mistake (dropped term, wrong sign, wrong index,
transposed operand) would break.
"""
import math
import os
from collections import deque

import numpy as np
import pytest

import lidarsim
import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# helpers that do NOT reuse the oracle's code
# --------------------------------------------------------------------------
def grid_scan(points_fn, H, W, elev=None):
    """Organized scan whose point (i, c) is points_fn(i, c); rows already top->bottom."""
    xyzr = np.zeros((H, W, 4), np.float32)
    for i in range(H):
        for c in range(W):
            x, y, z = points_fn(i, c)
            xyzr[i, c, :3] = (x, y, z)
            xyzr[i, c, 3] = math.sqrt(x * x + y * y + z * z)
    if elev is None:
        elev = np.linspace(0.2, -0.2, H).astype(np.float32) if H > 1 else np.zeros(1, np.float32)
    return xyzr, np.asarray(elev, np.float32)


def canon(lab):
    """Relabel a partition to the order of first appearance (-1/0 kept as background)."""
    out = np.full(lab.shape, -1, np.int64)
    mp = {}
    flat = lab.ravel()
    res = out.ravel()
    for k, v in enumerate(flat):
        if v < 0:
            continue
        if v not in mp:
            mp[v] = len(mp)
        res[k] = mp[v]
    return res.reshape(lab.shape)


def nb_edges_bruteforce(H, Ws, wrap):
    """All joined pairs by the paper's join statement, by enumerating vertex
    pairs: p(i,j) joins p(i+1,j), p(i+1,j+1), p(i,j+1); the last ring joins only
    horizontally; the last column joins column 0 (Sec. 2, mesh construction)."""
    wr = wrap and Ws >= 3
    pairs = {}
    for i1 in range(H):
        for j1 in range(Ws):
            for i2 in range(H):
                for j2 in range(Ws):
                    di = i2 - i1
                    dj = j2 - j1
                    if wr and j1 == Ws - 1 and j2 == 0:
                        dj = 1
                    if (di, dj) == (0, 1):
                        pairs[(i1, j1, i2, j2)] = "R"
                    elif (di, dj) == (1, 0):
                        pairs[(i1, j1, i2, j2)] = "D"
                    elif (di, dj) == (1, 1):
                        pairs[(i1, j1, i2, j2)] = "G"
    return pairs


BITS = {"R": O.BIT_R, "D": O.BIT_D, "G": O.BIT_G}
HBITS = {"R": O.BIT_HR, "D": O.BIT_HD, "G": O.BIT_HG}


def bfs_labels(mb, W, s, wrap):
    """Brute-force components from the explicit edge list (independent BFS)."""
    H, Ws = mb.shape
    adj = {(i, j): [] for i in range(H) for j in range(Ws)}
    for (i1, j1, i2, j2), kind in nb_edges_bruteforce(H, Ws, wrap).items():
        if mb[i1, j1] & HBITS[kind]:
            adj[(i1, j1)].append((i2, j2))
            adj[(i2, j2)].append((i1, j1))
    lab = np.full((H, Ws), -1, np.int64)
    verts = [(i, j) for i in range(H) for j in range(Ws) if mb[i, j] & O.BIT_VALID]
    for v in verts:
        if lab[v] != -1:
            continue
        comp = [v]
        seen = {v}
        q = deque([v])
        while q:
            u = q.popleft()
            for w in adj[u]:
                if w not in seen:
                    seen.add(w)
                    comp.append(w)
                    q.append(w)
        m = min(i * W + j * s for i, j in comp)
        for u in comp:
            lab[u] = m
    return lab


def random_mask(rng, H, Ws, wrap, p_valid=0.8, p_edge=0.8, p_homog=0.6):
    """Random consistent mesh bytes: homogeneous subset of mesh edges, which
    are a subset of the pairs joinable between valid vertices."""
    mb = np.zeros((H, Ws), np.uint8)
    valid = rng.random((H, Ws)) < p_valid
    mb[valid] |= O.BIT_VALID
    for (i1, j1, i2, j2), kind in nb_edges_bruteforce(H, Ws, wrap).items():
        if valid[i1, j1] and valid[i2, j2] and rng.random() < p_edge:
            mb[i1, j1] |= BITS[kind]
            if rng.random() < p_homog:
                mb[i1, j1] |= HBITS[kind]
    return mb


def params_for(spec, **kw):
    p = O.Params(subsample=spec.subsample, r_max=spec.r_max, jump_rel_h=spec.jump_rel_h,
                 jump_rel_v=spec.jump_rel_v, angle_rad=math.radians(spec.angle_deg))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v)


def ang(a, b):
    a = unit(a)
    b = unit(b)
    return math.atan2(np.linalg.norm(np.cross(a, b)), float(np.dot(a, b)))


# --------------------------------------------------------------------------
# step 1: decode
# --------------------------------------------------------------------------
def test_ring_order_matches_stable_descending_sort():
    rng = np.random.default_rng(5)
    for n in (1, 2, 7, 16, 64, 128):
        e = rng.choice(np.linspace(-0.4, 0.1, 9), size=n).astype(np.float32)  # ties included
        want = np.lexsort((np.arange(n), -e.astype(np.float64)))
        assert np.array_equal(O.ring_order(e), want)


def test_range_only_decode_is_spherical_to_cartesian():
    th = np.array([0.3, -0.1], np.float32)
    r = np.array([[2.0, 4.0, 0.0], [1.5, 3.0, 5.0]], np.float32)
    az0, daz = np.float32(0.25), np.float32(0.5)
    order, rs, xyz, valid = O.decode(th, az0, daz, None, r, 0.0, 4.5)
    for i in range(2):
        for c in range(3):
            t = float(th[i])
            phi = float(az0) + c * float(daz)
            want = float(r[i, c]) * np.array([math.cos(t) * math.cos(phi), math.cos(t) * math.sin(phi),
                                              math.sin(t)])
            assert np.allclose(xyz[i, c], want, rtol=0, atol=1e-15)
    assert valid.tolist() == [[1, 1, 0], [1, 1, 0]]  # r=0 dropout, r=5 > r_max


# --------------------------------------------------------------------------
# step 2: mesh
# --------------------------------------------------------------------------
@pytest.mark.parametrize("wrap", [0, 1])
def test_mesh_matches_bruteforce_join_rule(wrap):
    rng = np.random.default_rng(11 + wrap)
    for _ in range(150):
        H = int(rng.integers(1, 6))
        W = int(rng.integers(1, 9))
        s = int(rng.integers(1, 4))
        Ws = O.ws_of(W, s)
        rs = rng.uniform(1.0, 3.0, (H, W)).astype(np.float32)
        rs[rng.random((H, W)) < 0.2] = 0.0
        valid = (rs > 0).astype(np.uint8)
        mb = O.mesh(rs, valid, s, wrap, np.inf, np.inf)
        got = {}
        for (i1, j1, i2, j2), kind in nb_edges_bruteforce(H, Ws, wrap).items():
            want = bool(valid[i1, j1 * s] and valid[i2, j2 * s])
            got[(i1, j1, kind)] = want
            assert bool(mb[i1, j1] & BITS[kind]) == want
        # no other bits are set
        for i in range(H):
            for j in range(Ws):
                for kind in "RDG":
                    if (i, j, kind) not in got:
                        assert not mb[i, j] & BITS[kind]
                assert bool(mb[i, j] & O.BIT_VALID) == bool(valid[i, j * s])


def test_mesh_edge_counts_closed_form():
    H, W = 7, 12
    rs = np.full((H, W), 5.0, np.float32)
    v = np.ones((H, W), np.uint8)
    for wrap in (0, 1):
        mb = O.mesh(rs, v, 1, wrap, 0.1, 0.1)
        nR = int(((mb & O.BIT_R) > 0).sum())
        nD = int(((mb & O.BIT_D) > 0).sum())
        nG = int(((mb & O.BIT_G) > 0).sum())
        if wrap:
            assert (nR, nD, nG) == (H * W, (H - 1) * W, (H - 1) * W)
        else:
            assert (nR, nD, nG) == (H * (W - 1), (H - 1) * W, (H - 1) * (W - 1))
        # the last ring joins only horizontally
        assert not (mb[-1] & (O.BIT_D | O.BIT_G)).any()
        nbr, cnt = O.neighbours(mb, W, 1, wrap)
        assert cnt.max() == 6  # "six of them are connected" (Sec. 2)
        assert (cnt[1:-1, 1:-1] == 6).all()


def test_single_dropout_removes_its_six_edges():
    H, W = 5, 9
    rs = np.full((H, W), 5.0, np.float32)
    v = np.ones((H, W), np.uint8)
    full = O.mesh(rs, v, 1, 1, 0.1, 0.1)
    v2 = v.copy()
    v2[2, 4] = 0
    rs2 = rs.copy()
    rs2[2, 4] = 0
    holed = O.mesh(rs2, v2, 1, 1, 0.1, 0.1)
    cnt = lambda m: int(sum(((m & b) > 0).sum() for b in (O.BIT_R, O.BIT_D, O.BIT_G)))
    assert cnt(full) - cnt(holed) == 6


def test_depth_jump_cuts_only_across_the_step():
    H, W = 3, 8
    rs = np.full((H, W), 10.0, np.float32)
    rs[:, 4:] = 12.0  # 20 % relative jump between columns 3 and 4
    v = np.ones((H, W), np.uint8)
    cut = O.mesh(rs, v, 1, 0, 0.10, np.inf)
    keep = O.mesh(rs, v, 1, 0, 0.25, np.inf)
    assert not (cut[:, 3] & O.BIT_R).any()
    assert (cut[:, 2] & O.BIT_R).all() and (cut[:, 4] & O.BIT_R).all()
    assert (keep[:, 3] & O.BIT_R).all()
    # vertical edges across the step (G of column 3) obey jump_rel_v, here off
    assert (cut[:-1, 3] & O.BIT_G).all()
    vcut = O.mesh(rs, v, 1, 0, np.inf, 0.10)
    assert not (vcut[:-1, 3] & O.BIT_G).any() and (vcut[:-1, 3] & O.BIT_D).all()


def _pair_cut(r_p, r_q, tau):
    """Is the R edge of a 1 x 2 ring (ranges r_p, r_q) cut at threshold tau?
    And the D and G edges of a 2 x 2 grid whose top row is r_p and bottom row
    r_q, with the same threshold as jump_rel_v?"""
    rs = np.array([[r_p, r_q]], np.float32)
    mh = O.mesh(rs, np.ones((1, 2), np.uint8), 1, 0, tau, np.inf)
    rv = np.array([[r_p, r_p], [r_q, r_q]], np.float32)
    mv = O.mesh(rv, np.ones((2, 2), np.uint8), 1, 0, np.inf, tau)
    return (not (mh[0, 0] & O.BIT_R), not (mv[0, 0] & O.BIT_D), not (mv[0, 0] & O.BIT_G))


def test_depth_jump_threshold_scales_with_the_nearer_range():
    # cut <=> |r_p - r_q| > tau * min(r_p, r_q): ranges 10 and 12 differ by
    # exactly 2; tau = 0.18 gives 1.8 on the nearer range (cut) but 2.16 on
    # the farther one (kept), in either order of the two points
    assert _pair_cut(10.0, 12.0, 0.18) == (True, True, True)
    assert _pair_cut(12.0, 10.0, 0.18) == (True, True, True)
    # tau = 0.21: 2.1 on the nearer range, kept
    assert _pair_cut(10.0, 12.0, 0.21) == (False, False, False)


def test_depth_jump_at_the_threshold_is_kept():
    # strict '>': ranges 2 and 3 with tau = 0.5 give |dr| = 1 = tau * 2
    # exactly (binary32), which does not cut; a hair less cuts
    assert float(np.float32(0.5) * np.float32(2.0)) == 1.0
    assert _pair_cut(2.0, 3.0, 0.5) == (False, False, False)
    assert _pair_cut(3.0, 2.0, 0.5) == (False, False, False)
    assert _pair_cut(2.0, 3.0, float(np.nextafter(np.float32(0.5), np.float32(0)))) == (True, True, True)


def test_range_validity_bounds():
    # Sec. 2 "within range of the Lidar": r_min < r <= r_max; r at r_max is
    # in range, r at r_min is not
    r = np.array([[1.0, 2.0, 4.5, 4.50001]], np.float32)
    _, _, _, valid = O.decode(np.zeros(1, np.float32), 0.0, 0.1, None, r, 1.0, 4.5)
    assert valid.tolist() == [[0, 1, 1, 0]]


# --------------------------------------------------------------------------
# step 3: normals
# --------------------------------------------------------------------------
def _normals_of_grid(xyzr, elev, wrap=0, daz=0.01):
    p = O.Params(subsample=1, r_max=1e9, jump_rel_h=np.inf, jump_rel_v=np.inf, wrap=wrap)
    return O.segment(elev, 0.0, daz, xyzr, p)


def test_flat_ground_normal_is_exactly_up():
    # ground z=-2 seen by a sensor looking along +x: lower rings are nearer
    # (x decreases with i), later shots are further anticlockwise (y grows)
    xyzr, elev = grid_scan(lambda i, c: (10.0 - 0.5 * i, 0.25 * c - 1.0, -2.0), 5, 8)
    r = _normals_of_grid(xyzr, elev)
    has = (r.meshbits & O.BIT_HASN) > 0
    assert has.all()
    assert np.array_equal(r.normals[has], np.tile([0.0, 0.0, 1.0], (has.sum(), 1)))
    assert r.nseg == 1


def test_tilted_plane_normal_exact():
    f = lambda i, c: (10.0 - 0.5 * i, 0.25 * c - 1.0, -2.0 + 0.5 * (10.0 - 0.5 * i) + 0.25 * (0.25 * c - 1.0))
    xyzr, elev = grid_scan(f, 5, 8)
    r = _normals_of_grid(xyzr, elev)
    want = unit([-0.5, -0.25, 1.0])
    has = (r.meshbits & O.BIT_HASN) > 0
    assert has.all()
    assert np.abs(r.normals[has] - want).max() < 1e-15
    # mirrored spin direction flips the orientation convention back to the sensor side
    r2 = _normals_of_grid(xyzr[:, ::-1].copy(), elev, daz=-0.01)
    assert np.abs(r2.normals[has[:, ::-1]] - want).max() < 1e-15


def test_weighted_normal_hand_worked_example():
    """p=(0,0,0), A=(-2,0,0), B=(-2,1,0), C=(0,1,1) on a 2x2 grid (no wrap).
    Triangles AB and BC exist.  A x B = (0,0,-2), B x C = (1,2,-2);
    w_AB = 1/(|A|+|B|) = 1/(2+sqrt5) = sqrt5 - 2,
    w_BC = 1/(|B|+|C|) = 1/(sqrt5+sqrt2) = (sqrt5 - sqrt2)/3;
    n = -(w_AB (0,0,-2) + w_BC (1,2,-2)) / |.|  (Sec. 2, weighted average)."""
    pts = {(0, 0): (0, 0, 0), (1, 0): (-2, 0, 0), (1, 1): (-2, 1, 0), (0, 1): (0, 1, 1)}
    xyzr, elev = grid_scan(lambda i, c: pts[(i, c)], 2, 2)
    xyzr[0, 0, 3] = 1.0  # range of the origin point must be valid
    r = _normals_of_grid(xyzr, elev)
    w1 = math.sqrt(5) - 2
    w2 = (math.sqrt(5) - math.sqrt(2)) / 3
    want = unit([-w2, -2 * w2, 2 * w1 + 2 * w2])
    assert np.abs(r.normals[0, 0] - want).max() < 1e-14
    # the fixture separates the paper's weighting from nearby readings
    unweighted = unit([-1, -2, 4])
    assert ang(want, unweighted) > 1e-2
    # cut the rim edge A-B (horizontal depth jump): triangle AB no longer
    # counts although both of its spokes exist, so n = -(B x C)/|B x C|
    xyzr[1, 0, 3], xyzr[1, 1, 3], xyzr[0, 1, 3] = 1.0, 5.0, 1.0
    xyzr[0, 0, 3] = 1.0
    p = O.Params(subsample=1, r_max=1e9, jump_rel_h=0.1, jump_rel_v=np.inf, wrap=0)
    r2 = O.segment(elev, 0.0, 0.01, xyzr, p)
    assert r2.meshbits[1, 0] & O.BIT_R == 0 and r2.meshbits[0, 0] & (O.BIT_D | O.BIT_G) == O.BIT_D | O.BIT_G
    assert np.abs(r2.normals[0, 0] - np.array([-1.0, -2.0, 2.0]) / 3.0).max() < 1e-15
    assert r.kappa[0, 0] == pytest.approx((w1 * 2 * math.sqrt(5) + w2 * math.sqrt(5) * math.sqrt(2))
                                          / np.linalg.norm([w2, 2 * w2, -2 * w1 - 2 * w2]), rel=1e-14)


def test_isolated_and_collinear_vertices_have_no_normal():
    # one ring only: no triangles anywhere
    xyzr, elev = grid_scan(lambda i, c: (5.0, 0.1 * c, 0.0), 1, 6)
    r = _normals_of_grid(xyzr, elev)
    assert not (r.meshbits & O.BIT_HASN).any()
    assert r.nseg == 6  # every valid vertex is its own segment
    # all points on one line: triangles exist but every cross product is 0
    xyzr, elev = grid_scan(lambda i, c: (5.0 + 0.5 * i + 0.25 * c, 0.0, 0.0), 3, 4)
    r = _normals_of_grid(xyzr, elev)
    assert not (r.meshbits & O.BIT_HASN).any()


def test_inside_cylinder_normals_point_at_the_axis():
    # sensor on the axis of a vertical cylinder of radius 6: the surface seen
    # from inside faces the sensor, i.e. the normal is the inward radial
    spec = lidarsim.SceneSpec("cyl", lidarsim.elev_uniform(-10, 10, 9), 360, seed=1, sigma=0.0, p_drop=0.0,
                              r_max=100.0)
    prims = np.array([[lidarsim.PRIM_CYL, 1, 0.0, 0.0, 6.0, -50.0, 50.0, 0, 0, 0]])
    scan = lidarsim.raycast(spec, prims=prims)
    p = params_for(spec, subsample=1)
    r = O.segment_scan(scan, p, range_only=True)
    H, W = r.meshbits.shape
    dphi = scan.daz
    worst = 0.0
    for i in range(1, H - 1):
        for j in range(W):
            phi = scan.az0 + j * dphi
            want = [-math.cos(phi), -math.sin(phi), 0.0]
            worst = max(worst, ang(r.normals[i, j], want))
    assert worst < dphi  # chord triangles tilt by O(dphi); a wrong sign/index is O(1)
    assert r.nseg == 1


def test_ray_cast_ground_plane_is_one_segment():
    spec = lidarsim.ring16(seed=7)
    prims = lidarsim.scene_prims(lidarsim.SceneSpec("g", [0], 8, seed=7))[:1]  # ground only
    scan = lidarsim.raycast(spec, prims=prims, sigma=0.0, p_drop=0.0)
    # far ground rings are more than 2x apart in range: keep vertical joins
    p = params_for(spec, jump_rel_v=np.inf)
    for ro in (False, True):
        r = O.segment_scan(scan, p, range_only=ro)
        has = (r.meshbits & O.BIT_HASN) > 0
        assert r.nseg == 1
        errs = [ang(n, [0, 0, 1]) for n in r.normals[has]]
        assert max(errs) < 1e-4  # float32 rounding of the ray-cast points only


# --------------------------------------------------------------------------
# step 4: edge predicate
# --------------------------------------------------------------------------
def _two_vertex_mask(n0, n1, pred, thr, comp=(0.2, 0.2, 0.2)):
    mb = np.array([[O.BIT_VALID | O.BIT_HASN | O.BIT_R, O.BIT_VALID | O.BIT_HASN]], np.uint8)
    nrm = np.array([[n0, n1]], np.float64)
    out, margin = O.edge_mask(nrm, mb, 2, 1, 0, pred, thr, comp)
    return bool(out[0, 0] & O.BIT_HR), margin[0, 0, 0]


def test_angle_predicate_threshold():
    t = math.radians(10.0)
    for eps in (1e-6, 1e-3):
        for sgn, want in ((-1, True), (+1, False)):
            a = t + sgn * eps
            h, m = _two_vertex_mask([0, 0, 1], [math.sin(a), 0, math.cos(a)], O.PRED_ANGLE, t)
            assert h == want
            assert m == pytest.approx(-sgn * eps, abs=1e-12)


def test_predicates_are_strict_at_equality():
    # Algorithm 1 compares with a strict '<'.  Angle form: equal normals make
    # an angle of exactly 0, so a threshold of 0 admits nothing; orthogonal
    # axes make atan2(1, 0) = pi/2 exactly, so pi/2 admits nothing either
    assert O.angle([0, 0, 1], [0, 0, 1]) == 0.0
    h, m = _two_vertex_mask([0, 0, 1], [0, 0, 1], O.PRED_ANGLE, 0.0)
    assert not h and m == 0.0
    h, _ = _two_vertex_mask([0, 0, 1], [0, 0, 1], O.PRED_ANGLE, 1e-12)
    assert h
    assert O.angle([1, 0, 0], [0, 1, 0]) == math.pi / 2
    h, _ = _two_vertex_mask([1, 0, 0], [0, 1, 0], O.PRED_ANGLE, math.pi / 2)
    assert not h
    # component form: a difference of exactly the threshold (dyadic values,
    # exact in binary64) on any one axis fails; the other axes are far inside
    n0 = [0.0, 0.0, 1.0]
    n1 = [0.25, 0.125, 0.75]
    d = [0.25, 0.125, 0.25]
    for axis in range(3):
        comp = [1.0, 1.0, 1.0]
        comp[axis] = d[axis]
        h, m = _two_vertex_mask(n0, n1, O.PRED_COMPONENT, 0.0, comp)
        assert not h and m == 0.0
        comp[axis] = d[axis] * (1 + 2 ** -40)
        h, _ = _two_vertex_mask(n0, n1, O.PRED_COMPONENT, 0.0, comp)
        assert h


def test_component_predicate_is_strict_componentwise():
    # (Algorithm 1): |di| < I, |dj| < J, |dk| < K
    base = unit([0.3, 0.2, 1.0])
    for axis in range(3):
        for delta, want in ((0.2 - 1e-6, True), (0.2 + 1e-6, False)):
            other = base.copy()
            other[axis] += delta
            h, _ = _two_vertex_mask(base, other, O.PRED_COMPONENT, 0.0)
            assert h == want


# --------------------------------------------------------------------------
# step 5: labels
# --------------------------------------------------------------------------
def test_components_match_bfs_and_algorithm1_on_tiny_grids():
    rng = np.random.default_rng(2024)
    for case in range(600):
        H = int(rng.integers(1, 7))
        W = int(rng.integers(1, 9))
        s = int(rng.integers(1, 4))
        wrap = int(rng.integers(0, 2))
        Ws = O.ws_of(W, s)
        mb = random_mask(rng, H, Ws, wrap, p_homog=rng.uniform(0.2, 0.9))
        vl, n = O.components(mb, W, s, wrap)
        want = bfs_labels(mb, W, s, wrap)
        assert np.array_equal(vl, want), (case, H, W, s, wrap)
        assert n == len(set(want[want >= 0].tolist()))
        L, n1 = O.algorithm1(mb, W, s, wrap)
        assert n1 == n
        assert np.array_equal(canon(np.where(L > 0, L, -1)), canon(vl))


def test_labels_are_canonical_min_index_on_a_real_scan():
    spec = lidarsim.ring16()
    scan = lidarsim.make_scan(spec)
    r = O.segment_scan(scan, params_for(spec))
    lab = r.labels.ravel()
    ids = np.arange(lab.size)
    for L in np.unique(lab[lab >= 0]):
        members = ids[lab == L]
        assert members.min() == L


# --------------------------------------------------------------------------
# step 6: back-fill
# --------------------------------------------------------------------------
def _read_golden(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *vals = line.split()
            rows[k] = [int(v) for v in vals]
    return rows


def test_backfill_hand_worked_ring():
    g = _read_golden("backfill_ring.txt")
    W, s = len(g["valid"]), 4
    valid = np.array([g["valid"]], np.uint8)
    vl = np.array([g["vlabel"]], np.int32)
    assert list(O.backfill(valid, vl, W, s, 0)[0]) == g["nowrap"]
    assert list(O.backfill(valid, vl, W, s, 1)[0]) == g["wrap"]


@pytest.mark.parametrize("case", ["s2", "s4", "s4u", "s3w"])
def test_backfill_ties_between_different_labels(case):
    # Sec. 2, last paragraph: nearest labelled point along the sweep; equal
    # distances go to the earlier sampled column (fixture worked by hand)
    g = _read_golden("backfill_ties.txt")
    W, s = g[case + "_W"][0], g[case + "_s"][0]
    valid = np.array([g[case + "_valid"]], np.uint8)
    vl = np.array([g[case + "_vlabel"]], np.int32)
    assert len(g[case + "_valid"]) == W and vl.shape[1] == O.ws_of(W, s)
    assert list(O.backfill(valid, vl, W, s, 0)[0]) == g[case + "_nowrap"]
    assert list(O.backfill(valid, vl, W, s, 1)[0]) == g[case + "_wrap"]


# --------------------------------------------------------------------------
# whole path: scene pins and invariances
# --------------------------------------------------------------------------
def test_box_faces_get_one_label_each():
    spec = lidarsim.SceneSpec("box", lidarsim.elev_uniform(-15, 5, 24), 1800, seed=3, sigma=0.0, p_drop=0.0,
                              r_max=100.0)
    ground = [lidarsim.PRIM_PLANE, 0, 0, 0, 1, -1.7, 0, 0, 0, 0]
    # a tall box seen across its vertical edge: faces x=8 and y=4 and the
    # ground are visible; the lowest ring sees ground in front of the box
    box = [lidarsim.PRIM_BOX, 1, 8.0, 4.0, -1.7, 12.0, 8.0, 1.0, 0, 0]
    scan = lidarsim.raycast(spec, prims=np.array([ground, box], np.float64))
    r = O.segment_scan(scan, params_for(spec, angle_rad=math.radians(10), jump_rel_v=1.0))
    gt = scan.gt[r.order]
    H, W = gt.shape
    # vertices whose 2-ring lies on one face
    interior = np.zeros((H, W), bool)
    for i in range(2, H - 2):
        for c in range(W):
            cols = [(c + d) % W for d in range(-2, 3)]
            blk = gt[i - 2:i + 3][:, cols]
            interior[i, c] = gt[i, c] >= 0 and (blk == gt[i, c]).all()
    faces = {}
    for f in np.unique(gt[interior]):
        labs = np.unique(r.labels[interior & (gt == f)])
        if (interior & (gt == f)).sum() >= 10:
            assert len(labs) == 1, (f, labs)
            faces[f] = labs[0]
    assert len(faces) >= 3  # ground + at least two visible faces
    assert len(set(faces.values())) == len(faces)


def test_decimation_invariance():
    """Sub-sampling by s equals running s=1 on every s-th column (Sec. 2)."""
    spec = lidarsim.ring64(cols=512)
    scan = lidarsim.make_scan(spec)
    for s in (2, 3, 5):
        p = params_for(spec, subsample=s)
        a = O.segment_scan(scan, p)
        dec = scan.xyzr[:, ::s].copy()
        p1 = params_for(spec, subsample=1)
        b = O.segment(scan.elev, scan.az0, scan.daz * s, dec, p1)
        assert np.array_equal(a.meshbits, b.meshbits)
        assert np.array_equal(a.normals, b.normals)
        assert np.array_equal(canon(a.vlabel), canon(b.vlabel))


def test_cyclic_shift_and_ring_shuffle_invariance():
    spec = lidarsim.ring16()
    scan = lidarsim.make_scan(spec)
    p = params_for(spec)
    base = O.segment_scan(scan, p)
    k = 137
    shifted = np.roll(scan.xyzr, -k, axis=1)
    sh = O.segment(scan.elev, scan.az0, scan.daz, shifted, p)
    assert np.array_equal(np.roll(base.meshbits, -k, axis=1), sh.meshbits)
    assert np.array_equal(canon(np.roll(base.vlabel, -k, axis=1)), canon(sh.vlabel))
    perm = np.random.default_rng(0).permutation(scan.rings)
    sf = O.segment(scan.elev[perm], scan.az0, scan.daz, scan.xyzr[perm], p)
    assert np.array_equal(sf.meshbits, base.meshbits)
    assert np.array_equal(sf.labels, base.labels)
    assert np.array_equal(sf.normals, base.normals)


def test_empty_and_degenerate_shapes():
    p = O.Params()
    r = O.segment(np.zeros(0, np.float32), 0.0, 0.01, np.zeros((0, 0, 4), np.float32), p)
    assert r.nseg == 0
    # one point
    xyzr = np.array([[[1.0, 0.0, 0.0, 1.0]]], np.float32)
    r = O.segment(np.zeros(1, np.float32), 0.0, 0.01, xyzr, p)
    assert r.nseg == 1 and r.labels[0, 0] == 0
    # all dropouts
    xyzr = np.zeros((3, 5, 4), np.float32)
    r = O.segment(np.zeros(3, np.float32), 0.0, 0.01, xyzr, p)
    assert r.nseg == 0 and (r.labels == -1).all()


# --------------------------------------------------------------------------
# post-processing: segment sizes and small-segment removal (Sec. 2, last paragraph)
# --------------------------------------------------------------------------
def test_segment_stats_hand_worked():
    # two rings of 6 points; labels are smallest point indices of their segments
    lab = np.array([[0, 0, 0, -1, 4, 4],
                    [0, 7, 7, 7, 7, -1]], np.int32)
    out, sizes, _, kept = O.segment_stats(lab, 3)
    assert sizes[0] == 4 and sizes[4] == 2 and sizes[7] == 4 and sizes.sum() == 10
    assert kept == 2
    assert out.tolist() == [[0, 0, 0, -1, -1, -1], [0, 7, 7, 7, 7, -1]]
    out1, _, _, kept1 = O.segment_stats(lab, 1)
    assert kept1 == 3 and np.array_equal(out1, lab)


def test_segment_stats_on_a_scan_are_consistent():
    spec = lidarsim.ring16()
    scan = lidarsim.make_scan(spec)
    r = O.segment_scan(scan, params_for(spec))
    out, sizes, nsum, kept = O.segment_stats(r.labels, 5, normals=r.normals, meshbits=r.meshbits)
    labelled = r.labels >= 0
    assert sizes.sum() == labelled.sum()
    # every removed point belonged to a segment of fewer than 5 points
    removed = labelled & (out < 0)
    assert np.all(sizes[r.labels[removed]] < 5)
    assert kept == int(np.sum(sizes >= 5))
    # a normal sum is never longer than the number of vertices summed
    lens = np.linalg.norm(nsum, axis=1)
    assert np.all(lens <= sizes + 1e-9)
    assert kept <= r.nseg

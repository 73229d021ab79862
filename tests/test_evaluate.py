"""The edge-based accuracy protocol (Sec. 3) on hand-made grids."""
import numpy as np

from paper_2005_02704_gb300 import evaluate as E


def test_boundary_of_two_halves():
    ids = np.array([[1, 1, 2, 2],
                    [1, 1, 2, 2]])
    valid = np.ones_like(ids, bool)
    b = E.boundary(ids, valid)
    # columns 1|2 differ, and columns 3|0 differ across the wrap
    assert b.tolist() == [[True, True, True, True], [True, True, True, True]]
    ids = np.array([[1, 1, 1, 1], [2, 2, 2, 2], [2, 2, 2, 2]])
    b = E.boundary(ids, np.ones_like(ids, bool))
    assert b.tolist() == [[True] * 4, [True] * 4, [False] * 4]


def test_perfect_segmentation_scores_one_and_relabelling_does_not_matter():
    rng = np.random.default_rng(0)
    gt = np.repeat(np.repeat(rng.integers(0, 5, (4, 6)), 3, axis=0), 5, axis=1)
    pred = gt * 7 + 100  # same partition, other names
    r = E.edge_prf(pred, gt, radius=1)
    assert r.precision == 1.0 and r.recall == 1.0 and r.f1 == 1.0


def test_shifted_boundary_needs_dilation():
    gt = np.zeros((5, 20), int)
    gt[:, 10:] = 1
    pred = np.zeros((5, 20), int)
    pred[:, 12:] = 1  # boundary two shots off (the seam boundary 19|0 agrees)
    r1 = E.edge_prf(pred, gt, radius=1)
    assert r1.precision == 0.75 and r1.recall == 0.75
    assert E.edge_prf(pred, gt, radius=2).f1 == 1.0


def test_over_segmentation_lowers_precision_only():
    gt = np.zeros((6, 12), int)
    pred = np.zeros((6, 12), int)
    pred[:, 6:] = 1  # a cut the ground truth does not have
    r = E.edge_prf(pred, gt, radius=1)
    assert r.precision == 0.0 and r.recall == 1.0 and r.n_gt == 0

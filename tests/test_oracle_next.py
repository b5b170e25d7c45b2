"""Pins of the oracle's two optional Sec. 2 steps (the original SLIC's seed
perturbation and its L1 stopping test) against hand-derived results:
uniform images, an L1 cone whose gradient minima are known in closed form,
a border-clamp case worked by hand, hand-computed residuals, and the
stopping iteration against runs with a fixed iteration count."""
import numpy as np
import pytest

import oracle
from paper_1509_04232_gb300 import synth


def _grey(v):
    v = np.asarray(v, dtype=np.uint8)
    return np.repeat(v[..., None], 3, axis=-1)


# --- seed perturbation ---------------------------------------------------------

def test_perturbation_leaves_seeds_on_a_uniform_image():
    img = np.zeros((48, 64, 3), np.uint8)
    img[...] = (90, 140, 30)
    feat = oracle.convert(img)
    c0 = oracle.init_centres(feat, 16)
    c1, g, _ = oracle.perturb_seeds(feat, 16, c0)
    assert np.array_equal(c0, c1)        # G = 0 everywhere: nothing is strictly lower
    assert np.all(g == 0.0)


def test_perturbation_on_an_l1_cone():
    """RGB features v = 5 (|x - 8| + |y - 6|) on 32x32, S = 16. Central
    differences are 10 * sign away from the apex row/column and 0 on it, so
    G = 300 ([x != 8] + [y != 6]) per grey channel triple: 0 at the apex,
    300 on its row and column, 600 elsewhere. Seed pixels (floor of the cell
    midpoints 7.5 and 23.5) and their moves, worked by hand:
      (7, 7)   -> (8, 6), the apex (G 0);
      (23, 7)  -> (22, 6), first row-6 candidate in scan order (G 300);
      (7, 23)  -> (8, 22), first column-8 candidate in scan order (G 300);
      (23, 23) stays: all nine candidates have G 600."""
    ys, xs = np.mgrid[0:32, 0:32]
    img = _grey(5 * (np.abs(xs - 8) + np.abs(ys - 6)))
    feat = oracle.convert(img, oracle.RGB)
    c0 = oracle.init_centres(feat, 16)
    c1, g, _ = oracle.perturb_seeds(feat, 16, c0)
    want = {0: (8, 6, 0.0, 0.0), 1: (22, 6, 70.0, 300.0), 2: (8, 22, 80.0, 300.0)}
    for k, (x, y, v, gk) in want.items():
        assert tuple(c1[k, 3:5]) == (x, y)
        assert np.all(c1[k, :3] == v)
        assert c1[k, 5] == 0.0
        assert g[k] == gk
    assert np.array_equal(c1[3], c0[3])  # (23.5, 23.5) keeps its midpoint and colour
    assert g[3] == 600.0


def test_perturbation_clamps_at_the_border():
    """One seed on a 3x1 grey image [0, 10, 30], S = 3 (midpoint x = 1). With
    neighbours clamped: G(0) = 3*10^2 = 300, G(1) = 3*30^2 = 2700,
    G(2) = 3*20^2 = 1200, so the seed moves to x = 0."""
    img = _grey(np.array([[0, 10, 30]]))
    feat = oracle.convert(img, oracle.RGB)
    c0 = oracle.init_centres(feat, 3)
    assert tuple(c0[0, 3:5]) == (1.0, 0.0)
    c1, g, margin = oracle.perturb_seeds(feat, 3, c0)
    assert tuple(c1[0]) == (0.0, 0.0, 0.0, 0.0, 0.0, 0.0)
    assert g[0] == 300.0
    assert margin[0] == pytest.approx((1200.0 - 300.0) / 300.0)


def test_perturbation_moves_at_most_one_pixel_and_lowers_the_gradient():
    img = synth.voronoi_frame(96, 64, 20, 8.0, 77)
    feat = oracle.convert(img)
    c0 = oracle.init_centres(feat, 16)
    c1, g, _ = oracle.perturb_seeds(feat, 16, c0)
    moved = np.any(c1 != c0, axis=1)
    assert moved.any()
    d = np.abs(c1[moved, 3:5] - np.floor(c0[moved, 3:5]))
    assert np.all(d <= 1.0) and np.all(c1[moved, 3:5] == np.round(c1[moved, 3:5]))
    # a moved seed's colour is the feature vector of its new pixel
    for k in np.flatnonzero(moved):
        x, y = int(c1[k, 3]), int(c1[k, 4])
        assert np.array_equal(c1[k, :3], feat[y, x])


# --- stopping test -------------------------------------------------------------

def test_residual_hand_values():
    prev = np.zeros((2, 6))
    cur = np.zeros((2, 6))
    prev[0, 3:5] = (1.0, 2.0)
    cur[0, 3:5] = (1.5, 1.0)    # |0.5| + |-1.0| = 1.5
    prev[1, 3:5] = (10.0, 10.0)
    cur[1, 3:5] = (7.0, 10.25)  # 3 + 0.25 = 3.25
    cur[1, :3] = (50.0, -3.0, 9.0)  # colour changes do not count
    assert oracle.residual(prev, cur) == pytest.approx((1.5 + 3.25) / 2)
    assert oracle.residual(cur, cur) == 0.0


def test_uniform_image_stops_after_one_update():
    img = np.full((48, 64, 3), 120, np.uint8)
    r = oracle.slic(img, S=16, iterations=8, convergence=1e-9)
    assert r["iterations_run"] == 1     # a fixed point: the first update moves nothing
    fixed = oracle.slic(img, S=16, iterations=8)
    assert fixed["iterations_run"] == 8
    assert np.array_equal(r["labels"], fixed["labels"])


def test_stopping_iteration_matches_fixed_runs():
    """E of update i, from runs with i-1 and i fixed iterations; a threshold
    between E_3 and min(E_1, E_2) must stop after exactly 3 updates with the
    labels and centres of the 3-iteration run."""
    img = synth.voronoi_frame(160, 120, 25, 6.0, 11)
    runs = [oracle.slic(img, S=16, iterations=i, enforce_connectivity=False) for i in range(5)]
    E = [None] + [oracle.residual(runs[i - 1]["centres"], runs[i]["centres"]) for i in range(1, 5)]
    assert E[3] < min(E[1], E[2])
    eps = 0.5 * (E[3] + min(E[1], E[2]))
    r = oracle.slic(img, S=16, iterations=10, enforce_connectivity=False, convergence=eps)
    assert r["iterations_run"] == 3
    assert np.array_equal(r["labels"], runs[3]["labels"])
    assert np.array_equal(r["centres"], runs[3]["centres"])
    # and the residual itself: the positions' mean L1 move, computed directly
    direct = np.mean(np.abs(runs[3]["centres"][:, 3:5] - runs[2]["centres"][:, 3:5]).sum(axis=1))
    assert E[3] == pytest.approx(direct, rel=1e-12)


def test_convergence_zero_runs_every_iteration():
    img = synth.voronoi_frame(64, 48, 8, 6.0, 3)
    assert oracle.slic(img, S=16, iterations=4)["iterations_run"] == 4

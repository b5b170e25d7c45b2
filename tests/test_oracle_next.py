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


# --- component-based connectivity (the original SLIC's, scope row f4) ------------

def _first_occurrence_order(lab):
    """Labels in raster order of their first pixel."""
    _, idx = np.unique(lab.ravel(), return_index=True)
    return lab.ravel()[np.sort(idx)]


def test_components_small_island_joins_its_left_neighbour():
    lab = np.zeros((6, 6), np.int32)
    lab[2, 2:4] = 1                       # 2 pixels <= 16/4: merged into the left pixel's segment
    out, n = oracle.connectivity_components(lab, 4)
    assert n == 1 and np.all(out == 0)


def test_components_segment_at_the_origin_is_kept():
    lab = np.zeros((6, 6), np.int32)
    lab[0, 0:2] = 5                       # first segment in scan order, small but kept
    out, n = oracle.connectivity_components(lab, 4)
    want = np.ones((6, 6), np.int32)
    want[0, 0:2] = 0
    assert n == 2 and np.array_equal(out, want)


def test_components_chain_of_small_segments():
    """Row 0: R R A A B R ... (A, B small). A's first pixel has R on its left;
    B's has A: B joins A's final segment, which is R's."""
    lab = np.full((5, 8), 7, np.int32)
    lab[0, 2:4] = 1
    lab[0, 4] = 2
    out, n = oracle.connectivity_components(lab, 4)
    assert n == 1 and np.all(out == 0)


def test_components_column_zero_uses_the_upper_neighbour():
    lab = np.zeros((6, 6), np.int32)
    lab[:3, 3:] = 3                       # a large second segment (9 pixels)
    lab[4, 0] = 9                         # small, in column 0: joins the segment above
    out, n = oracle.connectivity_components(lab, 4)
    want = np.zeros((6, 6), np.int32)
    want[:3, 3:] = 1
    assert n == 2 and np.array_equal(out, want)


def test_components_disconnected_label_is_two_segments():
    lab = np.zeros((8, 8), np.int32)
    lab[:, 3:5] = 1                       # splits label 0 into two large parts
    out, n = oracle.connectivity_components(lab, 4)
    assert n == 3
    assert list(_first_occurrence_order(out)) == [0, 1, 2]
    assert np.all(out[:, :3] == 0) and np.all(out[:, 3:5] == 1) and np.all(out[:, 5:] == 2)


def test_components_huge_minimum_merges_everything_into_the_first():
    lab = np.random.default_rng(2).integers(0, 6, (20, 30)).astype(np.int32)
    out, n = oracle.connectivity_components(lab, 10**9)
    assert n == 1 and np.all(out == 0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_components_without_merging_is_connected_component_labelling(seed):
    """min_size 0: every 4-connected component of each label is one segment,
    as scipy.ndimage.label finds them, numbered in scan order."""
    from scipy import ndimage
    rng = np.random.default_rng(seed)
    lab = rng.integers(0, 4, (23, 31)).astype(np.int32)
    lab = np.repeat(np.repeat(lab, 2, axis=0), 3, axis=1)[:40, :70]  # blocky, with thin joins
    out, n = oracle.connectivity_components(lab, 0)
    total = 0
    for v in np.unique(lab):
        comp, k = ndimage.label(lab == v)   # default structure: 4-connectivity
        total += k
        for c in range(1, k + 1):
            assert len(np.unique(out[comp == c])) == 1
    assert n == total and len(np.unique(out)) == total
    assert list(_first_occurrence_order(out)) == list(range(total))


def test_whole_run_component_mode_applies_the_relabelling():
    img = synth.voronoi_frame(96, 64, 12, 8.0, 19)
    r = oracle.slic(img, S=8, iterations=3, enforce_connectivity=2)
    want, _ = oracle.connectivity_components(r["labels_pre"], 8 * 8 // 4)
    assert np.array_equal(r["labels"], want)

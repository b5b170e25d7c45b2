"""Pins of the FP64 oracle against facts that do not come from the oracle:
textbook colour values, hand-worked instances of Eq. (1), hand-built
connectivity maps, closed forms (uniform and block images, a single
superpixel, m -> infinity, m = 0), brute force on tiny images and library
routines (numpy bincount means, scipy distances)."""
import numpy as np
import pytest
from scipy.spatial.distance import cdist

import oracle
from paper_1509_04232_gb300 import synth

from _golden import connectivity_cases, eq1_examples, lab_reference_colours


# --- grid (Sec. 2: S = sqrt(N/K)) ---------------------------------------------

@pytest.mark.parametrize("W,H,K,S,exp", [
    (320, 240, 300, 0, (16, 20, 15)),     # 76800/300 = 256 -> S = 16
    (640, 480, 1200, 0, (16, 40, 30)),
    (1920, 1080, 0, 16, (16, 120, 68)),   # 1080/16 = 67.5 -> a partial last row
    (3840, 2160, 0, 8, (8, 480, 270)),
    (10, 7, 1, 0, (8, 2, 1)),             # sqrt(70) = 8.37 -> 8
    (5, 5, 1000, 0, (1, 5, 5)),           # S clamps to 1
])
def test_grid(W, H, K, S, exp):
    assert oracle.grid(W, H, K, S) == exp


def test_grid_rejects_invalid():
    with pytest.raises(ValueError):
        oracle.grid(0, 10, 5, 0)
    with pytest.raises(ValueError):
        oracle.grid(10, 10, 0, 0)


# --- colour conversion (Sec. 2 CIELAB, Sec. 3 "Image space conversion") -------

@pytest.mark.parametrize("rgb,lab,tol", lab_reference_colours())
def test_lab_reference_colours(rgb, lab, tol):
    got = oracle.convert(np.array([[rgb]], np.uint8))[0, 0]
    np.testing.assert_allclose(got, lab, atol=tol, rtol=0)


def test_lab_greys_are_neutral_and_monotone():
    g = np.arange(256, dtype=np.uint8)
    img = np.stack([g, g, g], axis=-1)[None]
    lab = oracle.convert(img)[0]
    assert np.max(np.abs(lab[:, 1:])) < 1e-9           # white point = row sums
    assert np.all(np.diff(lab[:, 0]) > 0)               # L strictly increasing
    assert abs(lab[0, 0]) < 1e-12 and abs(lab[255, 0] - 100.0) < 1e-9


def test_lab_alpha_channel_ignored():
    rng = np.random.default_rng(1)
    rgb = rng.integers(0, 256, (7, 9, 3), dtype=np.uint8)
    rgba = np.concatenate([rgb, rng.integers(0, 256, (7, 9, 1), dtype=np.uint8)], axis=-1)
    np.testing.assert_array_equal(oracle.convert(rgb), oracle.convert(rgba))


def test_rgb_and_xyz_feature_spaces():
    rgb = np.array([[[12, 200, 255], [255, 255, 255]]], np.uint8)
    np.testing.assert_array_equal(oracle.convert(rgb, oracle.RGB)[0, 0], [12, 200, 255])
    xyz_white = oracle.convert(rgb, oracle.XYZ)[0, 1]
    # D65 white of the sRGB matrix: (95.047, 100.000, 108.883), textbook.
    np.testing.assert_allclose(xyz_white, [95.047, 100.0, 108.883], atol=2e-3)


# --- initialisation (Sec. 3 "Cluster center initialisation") ------------------

def test_init_centres_positions_and_colour():
    rng = np.random.default_rng(2)
    feat = rng.normal(size=(20, 35, 3))
    S = 8
    c = oracle.init_centres(feat, S)
    assert c.shape == (5 * 3, 6)
    # Full cell (r=1, c=2): x in [16,23], y in [8,15] -> midpoint (19.5, 11.5).
    k = 1 * 5 + 2
    np.testing.assert_array_equal(c[k, 3:], [19.5, 11.5, 0.0])
    np.testing.assert_array_equal(c[k, :3], feat[11, 19])
    # Partial corner cell (r=2, c=4): x in [32,34], y in [16,19] -> (33, 17.5).
    k = 2 * 5 + 4
    np.testing.assert_array_equal(c[k, 3:], [33.0, 17.5, 0.0])
    np.testing.assert_array_equal(c[k, :3], feat[17, 33])


# --- assignment (Eq. 1, Sec. 3 "Finding the cluster associations") -----------

@pytest.mark.parametrize("ex", eq1_examples(), ids=lambda e: e["name"])
def test_eq1_worked_examples(ex):
    W, H = ex["W"], ex["H"]
    feat = np.zeros((H, W, 3))
    for p in ex["pixels"]:
        feat[p["y"], p["x"]] = p["lab"]
    labels, margin = oracle.assign(feat, ex["S"], ex["m"], np.array(ex["centres"]))
    for p in ex["pixels"]:
        assert labels[p["y"], p["x"]] == p["label"], p
        want = (p["D_second"] - p["D_best"]) / p["D_best"]
        assert margin[p["y"], p["x"]] == pytest.approx(want, rel=1e-9, abs=1e-12), p


def _window_mask(W, H, S):
    """mask[i, k]: centre k's cell lies in the 3x3 cells around pixel i's cell."""
    ns_c, ns_r = -(-W // S), -(-H // S)
    ys, xs = np.mgrid[0:H, 0:W]
    pcx, pcy = (xs // S).ravel(), (ys // S).ravel()
    kc = np.arange(ns_c * ns_r) % ns_c
    kr = np.arange(ns_c * ns_r) // ns_c
    return (np.abs(pcx[:, None] - kc[None]) <= 1) & (np.abs(pcy[:, None] - kr[None]) <= 1)


def _random_centres(rng, W, H, S):
    ns_c, ns_r = -(-W // S), -(-H // S)
    K = ns_c * ns_r
    c = np.zeros((K, 6))
    c[:, 0] = rng.uniform(0, 100, K)
    c[:, 1:3] = rng.uniform(-80, 80, (K, 2))
    kc, kr = np.arange(K) % ns_c, np.arange(K) // ns_c
    c[:, 3] = np.minimum(kc * S + rng.uniform(0, S, K), W - 1)
    c[:, 4] = np.minimum(kr * S + rng.uniform(0, S, K), H - 1)
    return c


@pytest.mark.parametrize("W,H,S,m,seed", [(13, 11, 3, 10.0, 0), (24, 20, 4, 5.0, 1),
                                           (48, 40, 8, 20.0, 2), (17, 48, 8, 10.0, 3),
                                           (9, 9, 4, 0.0, 4), (31, 7, 3, 40.0, 5)])
def test_assign_matches_brute_force(W, H, S, m, seed):
    """Brute force: distance from every pixel to EVERY centre (scipy cdist),
    masked to the 3x3 cell window, first argmin."""
    rng = np.random.default_rng(seed)
    feat = np.stack([rng.uniform(0, 100, (H, W)), rng.uniform(-80, 80, (H, W)),
                     rng.uniform(-80, 80, (H, W))], -1)
    cen = _random_centres(rng, W, H, S)
    labels, margin = oracle.assign(feat, S, m, cen)
    ys, xs = np.mgrid[0:H, 0:W]
    xy = np.stack([xs.ravel(), ys.ravel()], -1).astype(float)
    d_lab = cdist(feat.reshape(-1, 3), cen[:, :3])
    d_xy = cdist(xy, cen[:, 3:5])
    D = np.where(_window_mask(W, H, S), d_lab + (m / S) * d_xy, np.inf)
    want = np.argmin(D, axis=1)
    Ds = np.sort(D, axis=1)
    tie = (Ds[:, 1] - Ds[:, 0]) <= 1e-9 * np.maximum(Ds[:, 0], 1e-12)
    got = labels.ravel()
    assert np.all((got == want) | tie)
    np.testing.assert_allclose(margin.ravel(), (Ds[:, 1] - Ds[:, 0]) / np.maximum(Ds[:, 0], 1e-12),
                               rtol=1e-6, atol=1e-9)


def test_assign_spatial_limit_is_voronoi():
    """m -> infinity: the colour term vanishes relative to space; the label is
    the spatially nearest of the 9 window centres."""
    rng = np.random.default_rng(7)
    W, H, S = 40, 32, 8
    feat = rng.uniform(0, 100, (H, W, 3))
    cen = _random_centres(rng, W, H, S)
    labels, _ = oracle.assign(feat, S, 1e12, cen)
    ys, xs = np.mgrid[0:H, 0:W]
    d = cdist(np.stack([xs.ravel(), ys.ravel()], -1).astype(float), cen[:, 3:5])
    d = np.where(_window_mask(W, H, S), d, np.inf)
    np.testing.assert_array_equal(labels.ravel(), np.argmin(d, axis=1))


def test_assign_colour_only_when_m_zero():
    rng = np.random.default_rng(8)
    W, H, S = 40, 32, 8
    feat = rng.uniform(0, 100, (H, W, 3))
    cen = _random_centres(rng, W, H, S)
    labels, _ = oracle.assign(feat, S, 0.0, cen)
    d = cdist(feat.reshape(-1, 3), cen[:, :3])
    d = np.where(_window_mask(W, H, S), d, np.inf)
    np.testing.assert_array_equal(labels.ravel(), np.argmin(d, axis=1))


# --- update (Sec. 3 "Updating the cluster center") ----------------------------

def test_update_is_member_mean_and_keeps_empty_centres():
    rng = np.random.default_rng(9)
    H, W, K = 19, 23, 12
    feat = rng.normal(size=(H, W, 3)) * 30
    labels = rng.integers(0, K - 2, (H, W)).astype(np.int32)   # centres K-2, K-1 empty
    old = rng.normal(size=(K, 6))
    new = oracle.update(feat, labels, old)
    ys, xs = np.mgrid[0:H, 0:W]
    cnt = np.bincount(labels.ravel(), minlength=K)
    for j, v in enumerate([feat[..., 0], feat[..., 1], feat[..., 2], xs, ys]):
        s = np.bincount(labels.ravel(), weights=v.ravel().astype(float), minlength=K)
        np.testing.assert_allclose(new[:K - 2, j], s[:K - 2] / cnt[:K - 2], rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(new[:K - 2, 5], cnt[:K - 2])
    np.testing.assert_array_equal(new[K - 2:, :5], old[K - 2:, :5])
    np.testing.assert_array_equal(new[K - 2:, 5], 0.0)


# --- connectivity (Sec. 3 "Enforce connectivity") -----------------------------

@pytest.mark.parametrize("case", connectivity_cases(), ids=lambda c: c["name"])
def test_connectivity_hand_cases(case):
    p1 = oracle.connectivity_pass(case["in"])
    np.testing.assert_array_equal(p1, case["pass1"])
    np.testing.assert_array_equal(oracle.connectivity_pass(p1), case["pass2"])


# --- whole runs: closed forms and invariants (Sec. 4 stage order) -------------

@pytest.mark.parametrize("W,H,S", [(64, 48, 16), (40, 24, 8), (96, 32, 32)])
def test_uniform_image_is_a_fixed_point(W, H, S):
    """Uniform colour, S dividing W and H: each pixel's own-cell midpoint is
    strictly nearest, so labels are the grid cells and centres never move.
    (With a partial last cell this does not hold: its midpoint is nearer to
    the edge pixels of the cell before it.)"""
    img = np.full((H, W, 3), (90, 140, 200), np.uint8)
    r = oracle.slic(img, S=S, m=10, iterations=4, enforce_connectivity=True)
    ys, xs = np.mgrid[0:H, 0:W]
    cells = (ys // S) * r["ns_c"] + xs // S
    np.testing.assert_array_equal(r["labels"], cells)
    init = oracle.init_centres(oracle.convert(img), S)
    np.testing.assert_allclose(r["centres"][:, :5], init[:, :5], atol=1e-12)
    cnt = np.bincount(cells.ravel())
    np.testing.assert_array_equal(r["centres"][:, 5], cnt)


def test_block_image_recovers_blocks():
    """Cell-aligned blocks of very different colours: labels are the cells,
    centres carry the block colour and the cell midpoint."""
    S, nc, nr = 8, 5, 4
    rng = np.random.default_rng(10)
    cols = rng.permutation(np.array([(r, g, b) for r in (0, 120, 255) for g in (0, 120, 255)
                                     for b in (0, 120, 255)], np.uint8))[:nc * nr]
    img = np.zeros((nr * S, nc * S, 3), np.uint8)
    for k, c in enumerate(cols):
        img[(k // nc) * S:(k // nc + 1) * S, (k % nc) * S:(k % nc + 1) * S] = c
    r = oracle.slic(img, S=S, m=10, iterations=5)
    ys, xs = np.mgrid[0:nr * S, 0:nc * S]
    np.testing.assert_array_equal(r["labels"], (ys // S) * nc + xs // S)
    lab = oracle.convert(cols[None])[0]
    np.testing.assert_allclose(r["centres"][:, :3], lab, atol=1e-9)
    k = np.arange(nc * nr)
    np.testing.assert_allclose(r["centres"][:, 3], (k % nc) * S + (S - 1) / 2)
    np.testing.assert_allclose(r["centres"][:, 4], (k // nc) * S + (S - 1) / 2)


def test_single_superpixel_is_global_mean():
    img = synth.voronoi_frame(30, 20, 5, 8.0, 123)
    r = oracle.slic(img, S=64, m=10, iterations=3, enforce_connectivity=False)
    assert r["ns_c"] == r["ns_r"] == 1
    assert np.all(r["labels"] == 0)
    feat = oracle.convert(img)
    np.testing.assert_allclose(r["centres"][0, :3], feat.reshape(-1, 3).mean(0), rtol=1e-12)
    np.testing.assert_allclose(r["centres"][0, 3:], [14.5, 9.5, 600.0], rtol=1e-12)


@pytest.mark.parametrize("iters", [1, 3])
def test_run_invariants(iters):
    """Before connectivity every label lies in its pixel's 3x3 cell window,
    and the returned centres are the member means of the previous pass."""
    img = synth.small_image(1)[:96, :112]
    r_prev = oracle.slic(img, K=42, m=10, iterations=iters - 1, enforce_connectivity=False)
    r = oracle.slic(img, K=42, m=10, iterations=iters, enforce_connectivity=True)
    S, ns_c = r["S"], r["ns_c"]
    H, W = r["labels_pre"].shape
    ys, xs = np.mgrid[0:H, 0:W]
    lab = r["labels_pre"]
    assert np.all(np.abs(lab % ns_c - xs // S) <= 1) and np.all(np.abs(lab // ns_c - ys // S) <= 1)
    feat = oracle.convert(img)
    prev = r_prev["labels_pre"].ravel()
    K = r["centres"].shape[0]
    cnt = np.bincount(prev, minlength=K)
    nz = cnt > 0
    for j, v in enumerate([feat[..., 0], feat[..., 1], feat[..., 2], xs, ys]):
        s = np.bincount(prev, weights=v.ravel().astype(float), minlength=K)
        np.testing.assert_allclose(r["centres"][nz, j], s[nz] / cnt[nz], rtol=1e-12, atol=1e-12)
    # the driver applies exactly two connectivity passes after the last assignment
    twice = oracle.connectivity_pass(oracle.connectivity_pass(r["labels_pre"]))
    np.testing.assert_array_equal(r["labels"], twice)


def test_iterations_zero_uses_initial_centres():
    img = synth.small_image(2)
    r = oracle.slic(img, K=300, m=10, iterations=0, enforce_connectivity=False)
    init = oracle.init_centres(oracle.convert(img), r["S"])
    np.testing.assert_array_equal(r["centres"], init)


def test_init_centres_argument_is_used():
    img = synth.small_image(3)
    r1 = oracle.slic(img, K=300, m=10, iterations=2)
    r2 = oracle.slic(img, K=300, m=10, iterations=0, init_centres=r1["centres"])
    assign_only, _ = oracle.assign(oracle.convert(img), r1["S"], 10.0, r1["centres"])
    np.testing.assert_array_equal(r2["labels_pre"], assign_only)

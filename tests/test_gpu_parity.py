"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (written here, used throughout):
  features        |gpu - oracle| <= 1e-4 * max(1, |oracle|)
  one assignment  from identical FP32 inputs: labels equal, except pixels
                  whose oracle tie margin is < 1e-5 (relative)
  one update      from identical labels: centres within 1e-4 * max(1, |ref|)
  connectivity    bit-exact on identical label maps
  whole run       >= 99.5 % label agreement with the oracle
"""
import numpy as np
import pytest

import oracle
from paper_1509_04232_gb300 import synth

from _golden import connectivity_cases

pytestmark = pytest.mark.gpu

FEAT_TOL = 1e-4
CENTRE_TOL = 1e-4
MARGIN_EPS = 1e-5
AGREE_MIN = 0.995


def _t(a, dev="cuda"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _np(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _seg(pkg, W, H, **kw):
    return pkg.Segmenter(W, H, **kw)


def _close(got, ref, tol):
    return np.abs(got - ref) <= tol * np.maximum(1.0, np.abs(ref))


# --- conversion --------------------------------------------------------------

@pytest.mark.parametrize("cs", [0, 1, 2])
def test_convert_all_byte_values(slic_gpu, cs):
    rng = np.random.default_rng(0)
    img = rng.integers(0, 256, (61, 67, 3), dtype=np.uint8)
    img[0, :64, 0] = np.arange(64)  # include every byte value somewhere
    img[1, :64, 1] = np.arange(64, 128)
    img[2, :64, 2] = np.arange(128, 192)
    img[3, :64, 0] = np.arange(192, 256)
    seg = _seg(slic_gpu, 67, 61, S=8, color_space=cs)
    got = _np(seg.convert(_t(img))).transpose(1, 2, 0)
    ref = oracle.convert(img, cs)
    assert np.all(_close(got, ref, FEAT_TOL)), np.max(np.abs(got - ref))


def test_convert_rgba_ignores_alpha(slic_gpu):
    img = synth.voronoi_frame(45, 29, 6, 8.0, 5, channels=4)
    img[..., 3] = np.random.default_rng(1).integers(0, 256, img.shape[:2])
    seg = _seg(slic_gpu, 45, 29, S=8, in_channels=4)
    got = _np(seg.convert(_t(img))).transpose(1, 2, 0)
    assert np.all(_close(got, oracle.convert(img), FEAT_TOL))


# --- initialisation ----------------------------------------------------------

@pytest.mark.parametrize("W,H,S", [(320, 240, 16), (70, 45, 16), (33, 21, 8), (5, 3, 7)])
def test_init_centres(slic_gpu, W, H, S):
    img = synth.voronoi_frame(W, H, 5, 8.0, 7)
    seg = _seg(slic_gpu, W, H, S=S)
    feat = seg.convert(_t(img))
    got = _np(seg.init_centres(feat))
    ref = oracle.init_centres(oracle.convert(img), S)
    np.testing.assert_array_equal(got[:, 3:], ref[:, 3:])            # positions, count: exact
    assert np.all(_close(got[:, :3], ref[:, :3], FEAT_TOL))


# --- one assignment from identical inputs -------------------------------------

def _perturbed_centres(feat, S, seed):
    rng = np.random.default_rng(seed)
    c = oracle.init_centres(feat, S)
    c[:, 3] += rng.uniform(-S / 3, S / 3, len(c))
    c[:, 4] += rng.uniform(-S / 3, S / 3, len(c))
    c[:, :3] += rng.normal(0, 5, (len(c), 3))
    return c


@pytest.mark.parametrize("W,H,S,m", [(320, 240, 16, 10.0), (333, 257, 13, 10.0), (100, 75, 8, 20.0),
                                     (97, 61, 4, 5.0), (64, 64, 32, 0.0), (37, 23, 3, 40.0),
                                     (1920, 1080, 16, 10.0)])
def test_one_assignment_matches_oracle(slic_gpu, W, H, S, m):
    img = synth.voronoi_frame(W, H, 40, 8.0, 11)
    feat64 = oracle.convert(img)
    feat32 = feat64.astype(np.float32)
    cen32 = _perturbed_centres(feat64, S, 3).astype(np.float32)
    # identical inputs: both sides see the FP32-rounded features and centres
    labels_ref, margin = oracle.assign(feat32.astype(np.float64), S, m, cen32.astype(np.float64))
    seg = _seg(slic_gpu, W, H, S=S, m=m)
    got = _np(seg.assign(_t(feat32.transpose(2, 0, 1).copy()), _t(cen32)))
    bad = (got != labels_ref) & (margin >= MARGIN_EPS)
    assert not bad.any(), f"{bad.sum()} labels differ away from ties"


# --- one update from identical labels ----------------------------------------

@pytest.mark.parametrize("W,H,S", [(320, 240, 16), (333, 257, 13), (1920, 1080, 16)])
def test_one_update_matches_oracle(slic_gpu, W, H, S):
    img = synth.voronoi_frame(W, H, 40, 8.0, 12)
    feat32 = oracle.convert(img).astype(np.float32)
    cen = _perturbed_centres(feat32.astype(np.float64), S, 4)
    labels, _ = oracle.assign(feat32.astype(np.float64), S, 10.0, cen)
    ref = oracle.update(feat32.astype(np.float64), labels, cen)
    seg = _seg(slic_gpu, W, H, S=S)
    got = _np(seg.update(_t(feat32.transpose(2, 0, 1).copy()), _t(labels), _t(cen.astype(np.float32))))
    assert np.all(_close(got, ref, CENTRE_TOL)), np.max(np.abs(got - ref))
    np.testing.assert_array_equal(got[:, 5], ref[:, 5])


def test_update_keeps_empty_centres(slic_gpu):
    W, H, S = 64, 48, 16
    rng = np.random.default_rng(5)
    feat = rng.uniform(0, 100, (3, H, W)).astype(np.float32)
    labels = np.zeros((H, W), np.int32)     # everything in centre 0
    cen = rng.normal(size=(12, 6)).astype(np.float32)
    seg = _seg(slic_gpu, W, H, S=S)
    got = _np(seg.update(_t(feat), _t(labels), _t(cen)))
    np.testing.assert_array_equal(got[1:, :5], cen[1:, :5])
    np.testing.assert_array_equal(got[1:, 5], 0)
    assert got[0, 5] == W * H


# --- connectivity ------------------------------------------------------------

@pytest.mark.parametrize("case", connectivity_cases(), ids=lambda c: c["name"])
def test_connectivity_hand_cases(slic_gpu, case):
    seg = _seg(slic_gpu, case["W"], case["H"], S=1)
    p1 = seg.connectivity_pass(_t(case["in"]))
    np.testing.assert_array_equal(_np(p1), case["pass1"])
    np.testing.assert_array_equal(_np(seg.connectivity_pass(p1)), case["pass2"])


def test_connectivity_random_maps(slic_gpu):
    rng = np.random.default_rng(6)
    lab = rng.integers(0, 4, (131, 77)).astype(np.int32)
    seg = _seg(slic_gpu, 77, 131, S=1)
    np.testing.assert_array_equal(_np(seg.connectivity_pass(_t(lab))), oracle.connectivity_pass(lab))


# --- whole runs --------------------------------------------------------------

def _run_both(pkg, img, **kw):
    H, W, C = img.shape
    seg = _seg(pkg, W, H, in_channels=C, **kw)
    labels, centres = seg.segment(_t(img))
    ref = oracle.slic(img, K=kw.get("K", 0), S=kw.get("S", 0), m=kw.get("m", 10.0),
                      iterations=kw.get("iterations", 10), color_space=kw.get("color_space", 0),
                      enforce_connectivity=kw.get("enforce_connectivity", True))
    return _np(labels), _np(centres), ref, seg


@pytest.mark.parametrize("frame", range(5))
def test_whole_run_small_workload(slic_gpu, frame):
    """320x240, 40 regions, sigma 8; K=300, m=10, 10 iterations, CIELAB."""
    img = synth.small_image(frame)
    labels, centres, ref, seg = _run_both(slic_gpu, img, K=300, m=10.0, iterations=10)
    assert (seg.S, seg.ns_c, seg.ns_r) == (16, 20, 15)
    agree = np.mean(labels == ref["labels"])
    assert agree >= AGREE_MIN, agree
    close = _close(centres, ref["centres"], 1e-2)
    assert np.mean(close) >= 0.99


@pytest.mark.parametrize("W,H,kw", [
    (333, 257, dict(S=13, m=10.0, iterations=5)),
    (100, 75, dict(S=8, m=20.0, iterations=3)),
    (97, 61, dict(K=50, m=5.0, iterations=4, enforce_connectivity=False)),
    (640, 480, dict(K=1200, m=10.0, iterations=5)),
    (64, 40, dict(S=8, m=10.0, iterations=3, color_space=1)),
    (64, 40, dict(S=8, m=10.0, iterations=3, color_space=2)),
    (100, 80, dict(S=2, m=10.0, iterations=2)),      # window too big for private sums
    (64, 48, dict(S=1, m=10.0, iterations=1)),
    (96, 64, dict(S=3, m=10.0, iterations=3)),
])
def test_whole_run_ragged_and_variants(slic_gpu, W, H, kw):
    img = synth.voronoi_frame(W, H, 30, 6.0, 21)
    labels, _, ref, _ = _run_both(slic_gpu, img, **kw)
    assert np.mean(labels == ref["labels"]) >= AGREE_MIN


def test_whole_run_1080p(slic_gpu):
    """1920x1080, 400 regions, sigma 6, S=16, m=10, 5 iterations (the
    benchmark's per-frame configuration)."""
    img = synth.hd_image(0)
    labels, centres, ref, seg = _run_both(slic_gpu, img, S=16, m=10.0, iterations=5)
    assert seg.K_eff == 8160
    assert np.mean(labels == ref["labels"]) >= AGREE_MIN


@pytest.mark.parametrize("W,H,S,it", [(1, 1, 1, 2), (5, 3, 7, 1), (3, 17, 2, 2), (16, 16, 16, 3)])
def test_degenerate_sizes(slic_gpu, W, H, S, it):
    img = synth.voronoi_frame(W, H, 3, 8.0, 9)
    labels, centres, ref, _ = _run_both(slic_gpu, img, S=S, m=10.0, iterations=it)
    np.testing.assert_array_equal(labels, ref["labels"])
    assert np.all(_close(centres, ref["centres"], CENTRE_TOL))


def test_iterations_zero(slic_gpu):
    img = synth.small_image(0)
    labels, centres, ref, _ = _run_both(slic_gpu, img, K=300, m=10.0, iterations=0)
    assert np.mean(labels == ref["labels"]) >= 0.999
    np.testing.assert_array_equal(centres[:, 3:], ref["centres"][:, 3:])


def test_invariants_on_gpu_output(slic_gpu):
    """Pre-connectivity labels lie in the pixel's 3x3 cell window; the output
    centres are the FP64 member means of the previous assignment."""
    import torch
    img = synth.small_image(3)
    H, W, _ = img.shape
    seg_prev = _seg(slic_gpu, W, H, K=300, iterations=2, enforce_connectivity=False)
    seg = _seg(slic_gpu, W, H, K=300, iterations=3, enforce_connectivity=False)
    lab_prev, _ = seg_prev.segment(_t(img))
    lab, cen = seg.segment(_t(img))
    lab, cen, lab_prev = _np(lab), _np(cen), _np(lab_prev)
    S, ns_c = seg.S, seg.ns_c
    ys, xs = np.mgrid[0:H, 0:W]
    assert np.all(np.abs(lab % ns_c - xs // S) <= 1) and np.all(np.abs(lab // ns_c - ys // S) <= 1)
    feat = _np(seg.convert(_t(img))).astype(np.float64)
    K = seg.K_eff
    cnt = np.bincount(lab_prev.ravel(), minlength=K)
    nz = cnt > 0
    for j, v in enumerate([feat[0], feat[1], feat[2], xs, ys]):
        s = np.bincount(lab_prev.ravel(), weights=v.ravel().astype(float), minlength=K)
        assert np.all(_close(cen[nz, j], s[nz] / cnt[nz], CENTRE_TOL))
    np.testing.assert_array_equal(cen[:, 5], cnt)


def test_deterministic_and_launch_count(slic_gpu):
    img = synth.small_image(4)
    seg = _seg(slic_gpu, 320, 240, K=300, iterations=10)
    n0 = seg.launches
    l1, c1 = seg.segment(_t(img))
    n1 = seg.launches
    l2, c2 = seg.segment(_t(img))
    np.testing.assert_array_equal(_np(l1), _np(l2))
    np.testing.assert_array_equal(_np(c1), _np(c2))
    assert n1 - n0 == 2 * 10 + 4      # init, 11 assignments, 10 updates, 2 connectivity


def test_init_centres_override(slic_gpu):
    img = synth.small_image(2)
    ref1 = oracle.slic(img, K=300, m=10, iterations=2)
    seg = _seg(slic_gpu, 320, 240, K=300, iterations=0)
    init = _t(ref1["centres"].astype(np.float32))
    labels, centres = seg.segment(_t(img), init_centres=init)
    ref = oracle.slic(img, K=300, m=10, iterations=0, init_centres=ref1["centres"].astype(np.float32).astype(float))
    assert np.mean(_np(labels) == ref["labels"]) >= 0.999
    np.testing.assert_array_equal(_np(centres), ref1["centres"].astype(np.float32))


def test_profile_timers_single_frame(slic_gpu):
    """Assignment timers on a plain stream: one pair per assignment launch."""
    img = synth.small_image(2)
    seg = _seg(slic_gpu, 320, 240, K=300, iterations=4)
    slic_gpu.slic_profile_enable(seg.handle, True)
    seg.segment(_t(img))
    ms, n = slic_gpu.slic_profile_read(seg.handle)
    assert n == 5 and ms > 0

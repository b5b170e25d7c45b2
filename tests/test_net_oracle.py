"""Pins of the FP64 network oracle: central finite differences of the loss,
a one-layer case against an independent correlation (scipy), bfloat16
rounding against known bit patterns, slot <-> label round trips, and the
softmax cross-entropy gradient identities."""
import numpy as np
import pytest
from scipy.signal import correlate

from oracle import net_oracle as net


def _tiny(seed=0, H=7, W=9, S=4):
    rng = np.random.default_rng(seed)
    x0 = rng.normal(size=(H, W, net.C0))
    params = net.init_params(seed)
    valid = net.slot_mask(H, W, S)
    target = np.zeros((H, W), np.int64)
    for y in range(H):
        for x in range(W):
            target[y, x] = rng.choice(np.flatnonzero(valid[y, x]))
    return x0, params, target, valid


def test_bf16_rounding_bit_patterns():
    vals = np.array([1.0, 1.00390625, 1.005859375, 3.1415927, -2.5e-3, 65504.0], np.float32)
    r = net.bf16_round(vals)
    # bf16 keeps 8 significant bits: 1 + 2^-8 is a tie between 1 and 1 + 2^-7 -> even (1.0)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0078125
    assert r[3] == 3.140625
    assert np.all(np.abs(r - vals) <= np.abs(vals) * 2.0 ** -8)


@pytest.mark.parametrize("li,idx", [(0, (0, 1, 2, 3)), (1, (2, 2, 5, 7)), (2, (1, 0, 31, 0)),
                                    (3, (0, 2, 4, 8)), (3, "bias")])
def test_gradients_match_finite_differences(li, idx):
    x0, params, target, valid = _tiny()
    _, grads = net.backward(x0, params, target, valid, bf16=False)
    h = 1e-6
    p64 = [(w.astype(np.float64), b.astype(np.float64)) for w, b in params]

    def loss_with(delta):
        q = [(w.copy(), b.copy()) for w, b in p64]
        if idx == "bias":
            q[li][1][3] += delta
        else:
            q[li][0][idx] += delta
        return net.loss(net.forward(x0, q, bf16=False)[0], target, valid)

    num = (loss_with(h) - loss_with(-h)) / (2 * h)
    ana = grads[li][1][3] if idx == "bias" else grads[li][0][idx]
    assert ana == pytest.approx(num, rel=1e-6, abs=1e-10)


def test_one_layer_conv_is_a_correlation():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(6, 8, 3))
    w = rng.normal(size=(3, 3, 3, 2))
    b = rng.normal(size=2)
    out = net.conv3x3(x, w, b)
    for o in range(2):
        ref = sum(correlate(x[..., i], w[:, :, i, o], mode="same") for i in range(3)) + b[o]
        np.testing.assert_allclose(out[..., o], ref, rtol=1e-12, atol=1e-12)


def test_softmax_ce_gradient_identities():
    """dL/dlogits sums to zero per pixel, is zero on off-grid slots, and the
    loss of uniform logits is the mean log of the valid-slot count."""
    x0, params, target, valid = _tiny(1)
    H, W, _ = valid.shape
    logits = np.zeros((H, W, 9))
    assert net.loss(logits, target, valid) == pytest.approx(np.mean(np.log(valid.sum(-1))))
    # last-layer bias gradient = sum over pixels of (p - onehot) / (H W)
    _, grads = net.backward(x0, params, target, valid, bf16=False)
    lg, _ = net.forward(x0, params, bf16=False)
    p = np.where(valid, np.exp(net.masked_log_softmax(lg, valid)), 0.0)
    onehot = np.eye(9)[target]
    np.testing.assert_allclose(grads[3][1], (p - onehot).sum((0, 1)) / (H * W), atol=1e-12)
    assert abs(grads[3][1].sum()) < 1e-12


def test_slots_labels_round_trip():
    rng = np.random.default_rng(4)
    H, W, S = 20, 27, 6
    ns_c, ns_r = -(-W // S), -(-H // S)
    ys, xs = np.mgrid[0:H, 0:W]
    dy = rng.integers(-1, 2, (H, W))
    dx = rng.integers(-1, 2, (H, W))
    cy = np.clip(ys // S + dy, 0, ns_r - 1)
    cx = np.clip(xs // S + dx, 0, ns_c - 1)
    labels = (cy * ns_c + cx).astype(np.int32)
    slots = net.slots_from_labels(labels, S)
    np.testing.assert_array_equal(net.labels_from_slots(slots, S), labels)
    assert np.all(net.slot_mask(H, W, S)[ys, xs, slots])


def test_input_channels():
    lab = np.zeros((3, 5, 3))
    lab[..., 0] = 50.0
    lab[..., 1] = 64.0
    lab[..., 2] = -128.0
    x = net.input_channels(lab, 4)
    np.testing.assert_allclose(x[0, 0, :5], [0.5, 0.5, -1.0, 0.0, 0.0])
    np.testing.assert_allclose(x[2, 4, :5], [0.5, 0.5, -1.0, 0.0, 0.5])


def test_grid_distances_uniform_image():
    """Uniform colour: D is (m/S) times the distance to each grid midpoint
    (hand values for an 8x8 image, S=4, m=8: midpoints at 1.5 and 5.5)."""
    lab = np.full((8, 8, 3), 42.0)
    D = net.grid_distances(lab, 4, 8.0)
    # pixel (0,0): own centre (1.5,1.5) -> 2*sqrt(4.5); right centre (5.5,1.5) -> 2*sqrt(32.5)
    assert D[0, 0, 4] == pytest.approx(2 * np.sqrt(4.5))
    assert D[0, 0, 5] == pytest.approx(2 * np.sqrt(32.5))
    assert D[0, 0, 8] == pytest.approx(2 * np.sqrt(60.5))
    assert np.isinf(D[0, 0, [0, 1, 2, 3, 6]]).all()
    x = net.input_channels(lab, 4, 8.0)
    assert x[0, 0, 5 + 0] == 2.0 and x[0, 0, 5 + 4] == pytest.approx(2 * np.sqrt(4.5) / 100)

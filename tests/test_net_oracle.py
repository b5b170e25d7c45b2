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


# --- hand-worked forward cases (values below are worked out by hand) ------------

def _taps(cin, cout, centre, left=None, right=None, other=0.0):
    """A [3,3,cin,cout] kernel: `centre`, `left` (input x-1) and `right`
    (input x+1) taps of the middle kernel row as {(ci, co): value}; every
    other tap set to `other`."""
    w = np.full((3, 3, cin, cout), other)
    w[1, :, :, :] = 0.0 if other == 0.0 else other
    w[1, 0] = 0.0
    w[1, 1] = 0.0
    w[1, 2] = 0.0
    for dx, taps in ((0, left), (1, centre), (2, right)):
        for (ci, co), v in (taps or {}).items():
            w[1, dx, ci, co] = v
    return w


def test_forward_two_layers_relu_between_not_on_logits():
    """A 1x2 image through two layers. Layer 1 (1 -> 2 channels):
    z1 = (x[p] + 0.5 x[p+1] - 1.5, -x[p] + 0.5); with x = (1, 2):
    z1(0) = (1 + 1 - 1.5, -1 + 0.5) = (0.5, -0.5), z1(1) = (2 + 0 - 1.5, -2 + 0.5) = (0.5, -1.5),
    ReLU -> a1(0) = a1(1) = (0.5, 0). Layer 2 (2 -> 2): logit0 = a1_0[p] + 3 a1_1[p]
    + 2 a1_0[p-1] + 0.25, logit1 = -2 a1_0[p]:
    logits(0) = (0.5 + 0 + 0 + 0.25, -1) = (0.75, -1), logits(1) = (0.5 + 0 + 1 + 0.25, -1) = (1.75, -1).
    Without the ReLU logit0(0) would be 0.5 - 1.5 + 0.25 = -0.75; a ReLU on
    the logits would make logit1 zero."""
    x0 = np.array([[[1.0], [2.0]]])
    w1 = _taps(1, 2, centre={(0, 0): 1.0, (0, 1): -1.0}, right={(0, 0): 0.5})
    w2 = _taps(2, 2, centre={(0, 0): 1.0, (1, 0): 3.0, (0, 1): -2.0}, left={(0, 0): 2.0})
    params = [(w1, np.array([-1.5, 0.5])), (w2, np.array([0.25, 0.0]))]
    for bf16 in (False, True):  # every value here is a bfloat16 number
        logits, _ = net.forward(x0, params, bf16=bf16)
        np.testing.assert_array_equal(logits, [[[0.75, -1.0], [1.75, -1.0]]])


def test_forward_four_layers_relu_after_each_hidden_layer():
    """A 1x1 image (only centre taps see data: the other taps, set to 7, see
    the zero padding) through four layers 1 -> 2 -> 2 -> 2 -> 1:
    z1 = (a0, -a0) = (1, -1) -> a1 = (1, 0);
    z2 = (a1_0 + a1_1, a1_0 + 2 a1_1 - 3) = (1, -2) -> a2 = (1, 0);
    z3 = (a2_0 + a2_1 - 0.5, -a2_0) = (0.5, -1) -> a3 = (0.5, 0);
    logit = a3_0 + a3_1 - 1 = -0.5.
    Dropping the ReLU after layer 1, 2 or 3 gives -1, -1 or -1.5; a ReLU on
    the logit gives 0."""
    x0 = np.array([[[1.0]]])
    params = [
        (_taps(1, 2, centre={(0, 0): 1.0, (0, 1): -1.0}, other=7.0), np.array([0.0, 0.0])),
        (_taps(2, 2, centre={(0, 0): 1.0, (1, 0): 1.0, (0, 1): 1.0, (1, 1): 2.0}, other=7.0), np.array([0.0, -3.0])),
        (_taps(2, 2, centre={(0, 0): 1.0, (1, 0): 1.0, (0, 1): -1.0}, other=7.0), np.array([-0.5, 0.0])),
        (_taps(2, 1, centre={(0, 0): 1.0, (1, 0): 1.0}, other=7.0), np.array([-1.0])),
    ]
    for bf16 in (False, True):
        logits, _ = net.forward(x0, params, bf16=bf16)
        assert logits.shape == (1, 1, 1) and logits[0, 0, 0] == -0.5


def test_forward_bf16_rounding_points():
    """Where the precision model rounds to bfloat16 (8 significant bits; the
    spacing above 1 is 2^-7): the input channels, the weights and the
    activations stored between layers, but neither the biases nor the
    logits. v = 1 + 3*2^-9 = 1.005859375 lies 3/4 of a spacing above 1, so it
    rounds to 1 + 2^-7 = 1.0078125. On a 1x1 image with one channel:
      input v, weight 1, bias 0          -> logit 1.0078125 (input rounded)
      input 1, weight v, bias 0          -> logit 1.0078125 (weight rounded)
      input 1, weight 1, bias 3*2^-9, then a second layer of weight 1
                                         -> logit 1.0078125 (activation rounded)
      input 1, weight 1, bias 3*2^-9     -> logit 1.005859375 (bias, logit kept)"""
    v = 1.0 + 3 * 2.0 ** -9
    one = lambda w: _taps(1, 1, centre={(0, 0): w})  # noqa: E731
    cases = [
        (v, [(one(1.0), np.array([0.0]))], 1.0078125),
        (1.0, [(one(v), np.array([0.0]))], 1.0078125),
        (1.0, [(one(1.0), np.array([3 * 2.0 ** -9])), (one(1.0), np.array([0.0]))], 1.0078125),
        (1.0, [(one(1.0), np.array([3 * 2.0 ** -9]))], 1.005859375),
    ]
    for x, params, want in cases:
        got, _ = net.forward(np.array([[[x]]]), params, bf16=True)
        assert got[0, 0, 0] == want
        exact, _ = net.forward(np.array([[[x]]]), params, bf16=False)
        assert exact[0, 0, 0] == pytest.approx(1.005859375, abs=1e-15)


def test_backward_bf16_gradient_rounding_points():
    """The stored dL/dz of the bf16_grad model, on a 1x2 image with S = 1
    (two cells): pixel 0 may take slots 4 (own) and 5 (right), pixel 1 slots
    3 (left) and 4. Layer 1 gives hidden channel 0 the constant activation 1
    (bias 1); layer 2 has weight 1.25 from it to slot 5 (centre tap) and
    biases ln 2 on slot 3 and ln 2 - 1.25 on slot 5, so the logits are ln 2
    on slots 3 and 5 and 0 elsewhere. Targets: slot 4 at both pixels.
    Softmax: pixel 0 has p4 = 1/3, p5 = 2/3; pixel 1 has p3 = 2/3, p4 = 1/3.
    Mean-loss gradients (two pixels): dz4 = (1/3 - 1)/2 = -1/3, dz5 = dz3 = 1/3.
    1/3 in bfloat16 is 0.333984375 (1.0101011b x 2^-2), so the last layer's
    bias gradient is (1/3, -2/3, 1/3) exactly and (0.333984375, -0.66796875,
    0.333984375) with rounding. Hidden gradient at pixel 0: 1.25 dz5 =
    0.41666.. exactly; 1.25 x 0.333984375 = 0.41748046875 rounds to
    0.41796875 (1.671875 x 2^-2); pixel 1 has none (p5 = 0 there). So the
    first layer's bias gradient is 0.41666.. / 0.41796875."""
    x0 = np.zeros((1, 2, 1))
    w1 = _taps(1, 1, centre={})
    w2 = _taps(1, net.N_SLOTS, centre={(0, 5): 1.25})
    b2 = np.zeros(net.N_SLOTS)
    b2[3] = np.log(2.0)
    b2[5] = np.log(2.0) - 1.25
    params = [(w1, np.array([1.0])), (w2, b2)]
    valid = net.slot_mask(1, 2, 1)
    assert valid[0, 0].tolist() == [False] * 4 + [True, True] + [False] * 3
    assert valid[0, 1].tolist() == [False] * 3 + [True, True] + [False] * 4
    target = np.array([[4, 4]])
    _, g = net.backward(x0, params, target, valid, bf16=True, bf16_grad=False)
    np.testing.assert_allclose(g[1][1][3:6], [1 / 3, -2 / 3, 1 / 3], rtol=1e-12)
    assert g[0][1][0] == pytest.approx(1.25 / 3, rel=1e-12)
    _, g = net.backward(x0, params, target, valid, bf16=True, bf16_grad=True)
    np.testing.assert_array_equal(g[1][1][3:6], [0.333984375, -0.66796875, 0.333984375])
    assert g[0][1][0] == 0.41796875

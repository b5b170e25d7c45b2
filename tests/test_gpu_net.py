"""The warm-start network's CUDA kernels against the FP64 network oracle.

Tolerances (derived from the precision model: bf16 weights and stored
activations, FP32 accumulation vs FP64 in the oracle):
  logits     |gpu - oracle| <= 2e-2 * max(1, max |oracle|), and the argmax
             slot agrees wherever the oracle's top two logits differ by > 2e-2
  gradients  per element, |gpu - oracle| <= 2^-6 |oracle| + 2^-8 T + 2^-14 T1
             against the oracle with the device's bf16 gradient storage, T =
             the sum of the absolute values of the element's terms, T1 that
             of their FP32 summation scale
"""
import numpy as np
import pytest

import oracle
from oracle import net_oracle as NO
from paper_1509_04232_gb300 import synth

pytestmark = pytest.mark.gpu


def _split(flat):
    out, off = [], 0
    for cin, cout in NO.LAYERS:
        w = flat[off:off + 9 * cin * cout].reshape(3, 3, cin, cout)
        off += 9 * cin * cout
        b = flat[off:off + cout]
        off += cout
        out.append((w.astype(np.float64), b.astype(np.float64)))
    return out


def _setup(slic_gpu, n=2, W=48, H=40, S=8, seed=3):
    import torch
    from paper_1509_04232_gb300.warmstart import WarmStartNet
    net = WarmStartNet(W, H, S, max_batch=n, seed=seed)
    host = np.stack([synth.voronoi_frame(W, H, 12, 8.0, 900 + i) for i in range(n)])
    return net, host, torch.from_numpy(host).cuda()


def _oracle_input(img, S):
    return NO.input_channels(oracle.convert(img), S, 10.0)


def test_forward_matches_oracle(slic_gpu):
    import torch
    net, host, imgs = _setup(slic_gpu)
    logits = torch.empty((2, 40, 48, 16), dtype=torch.float32, device="cuda")
    labels = torch.empty((2, 40, 48), dtype=torch.int32, device="cuda")
    net.forward(imgs, logits=logits, labels=labels)
    torch.cuda.synchronize()
    net.status()
    params = _split(net.params())
    for i in range(2):
        ref, _ = NO.forward(_oracle_input(host[i], 8), params, bf16=True)
        got = logits[i].cpu().numpy()[..., :9]
        scale = max(1.0, np.abs(ref).max())
        assert np.max(np.abs(got - ref)) <= 2e-2 * scale
        valid = NO.slot_mask(40, 48, 8)
        z = np.where(valid, ref, -np.inf)
        top2 = np.sort(z, axis=-1)[..., -2:]
        clear = (top2[..., 1] - top2[..., 0]) > 2e-2 * scale
        want = NO.labels_from_slots(np.argmax(z, axis=-1), 8)
        assert np.all((labels[i].cpu().numpy() == want) | ~clear)
        assert np.all(logits[i].cpu().numpy()[..., 9:] == 0.0)


def test_forward_spans_several_tensor_core_tiles(slic_gpu):
    """A 300-pixel-wide image: rows of three 128-pixel tensor-core tiles, the
    last one ragged, in a batch of two."""
    import torch
    net, host, imgs = _setup(slic_gpu, n=2, W=300, H=21, S=12, seed=5)
    logits = torch.empty((2, 21, 300, 16), dtype=torch.float32, device="cuda")
    net.forward(imgs, logits=logits)
    torch.cuda.synchronize()
    net.status()
    params = _split(net.params())
    for i in range(2):
        ref, _ = NO.forward(_oracle_input(host[i], 12), params, bf16=True)
        got = logits[i].cpu().numpy()[..., :9]
        assert np.max(np.abs(got - ref)) <= 2e-2 * max(1.0, np.abs(ref).max())


def test_fused_labels_equal_labels_from_logits(slic_gpu):
    """The labels-only forward (argmax fused into the last tensor-core layer)
    gives the labels computed from the stored logits."""
    import torch
    net, host, imgs = _setup(slic_gpu, n=2, W=300, H=37, S=12, seed=6)
    logits = torch.empty((2, 37, 300, 16), dtype=torch.float32, device="cuda")
    want = torch.empty((2, 37, 300), dtype=torch.int32, device="cuda")
    got = torch.empty_like(want)
    net.forward(imgs, logits=logits, labels=want)
    net.forward(imgs, labels=got)
    torch.cuda.synchronize()
    net.status()
    assert torch.equal(got, want)


def _term_magnitudes(dzs, params):
    """Per layer (Tw, Tb, T1w, T1b). Tw, Tb: for every gradient element the
    sum of the absolute values of its terms, |a_in dz| (dW) and |dz| (db),
    with the oracle's stored dL/dz of the layer. T1w, T1b: the same with dz
    replaced by the scale of its own FP32 summation -- sum |dz_next| |w| over
    the next layer's taps for a hidden layer, 1/(H W) for the softmax
    gradient -- against which FP32-vs-FP64 noise of a near-cancelling dz is
    measured."""
    out = []
    L = len(dzs)
    for l, (dz, a_in) in enumerate(dzs):
        H, W, _ = dz.shape
        if l == L - 1:
            scale = np.full(dz.shape, 1.0 / (H * W))
        else:
            nxt = np.pad(np.abs(dzs[l + 1][0]), ((1, 1), (1, 1), (0, 0)))
            wq = np.abs(NO.bf16_round(params[l + 1][0]))
            scale = np.zeros(dz.shape)
            for dy in range(3):
                for dx in range(3):
                    scale += nxt[2 - dy:2 - dy + H, 2 - dx:2 - dx + W, :] @ wq[dy, dx].T
        ap = np.pad(np.abs(a_in), ((1, 1), (1, 1), (0, 0)))
        tw = np.zeros((3, 3, a_in.shape[2], dz.shape[2]))
        t1 = np.zeros_like(tw)
        for dy in range(3):
            for dx in range(3):
                win = ap[dy:dy + H, dx:dx + W, :]
                tw[dy, dx] = np.einsum("yxi,yxo->io", win, np.abs(dz))
                t1[dy, dx] = np.einsum("yxi,yxo->io", win, scale)
        out.append((tw, np.abs(dz).sum(axis=(0, 1)), t1, scale.sum(axis=(0, 1))))
    return out


def test_gradients_match_oracle(slic_gpu):
    """Every weight and bias gradient element against the FP64 oracle with
    dL/dz rounded to bf16 where the device stores it (bf16_grad). Two 160x80
    images: 400 weight-gradient tiles of 16x4 pixels, more than the 304
    persistent CTAs, so CTAs accumulate several tiles. What remains is FP32
    against FP64 summation and stored values that land on the other side of
    a bf16 rounding boundary: in the forward pass a few activations, whose
    one-step (2^-8 relative) changes move the logits and so every softmax
    gradient a little, each of which can again round either way. Each term
    is then off by at most about one bf16 step, so per element
        |gpu - oracle| <= 2^-6 |oracle| + 2^-8 T + 2^-14 T1,
    T = the sum of the absolute values of the element's terms (|a_in dz|
    over the pixels, with the oracle's stored dz) and T1 the same with dz
    replaced by the scale of the FP32 sum that produced it (a dz that nearly
    cancels carries FP32 noise of about 2^-24 times that scale per term). A
    wrong tap, channel or sign in one element moves it by about |g|, which
    is typically a tenth of T or more here (random targets): ten times the
    bound or more."""
    import torch
    n, W, H, S = 2, 160, 80, 8
    net, host, imgs = _setup(slic_gpu, n=n, W=W, H=H, S=S)
    rng = np.random.default_rng(0)
    valid = NO.slot_mask(H, W, S)
    target = np.zeros((n, H, W), np.uint8)
    for i in range(n):
        for y in range(H):
            for x in range(W):
                target[i, y, x] = rng.choice(np.flatnonzero(valid[y, x]))
    stats = torch.zeros(2, dtype=torch.float32, device="cuda")
    net.gradients(imgs, torch.from_numpy(target).cuda(), stats)
    torch.cuda.synchronize()
    g_gpu = _split(net.grads())
    params = _split(net.params())
    # the batch loss is the mean over the images: average the oracle's per-image gradients
    g_ref = [(np.zeros_like(w), np.zeros_like(b)) for w, b in params]
    t_ref = [(np.zeros_like(w), np.zeros_like(b)) for w, b in params]
    t1_ref = [(np.zeros_like(w), np.zeros_like(b)) for w, b in params]
    loss_ref = 0.0
    for i in range(n):
        x0 = _oracle_input(host[i], S)
        ti = target[i].astype(np.int64)
        li, gi, dzs = NO.backward(x0, params, ti, valid, bf16=True, bf16_grad=True, return_dz=True)
        mi = _term_magnitudes(dzs, params)
        loss_ref += li / n
        for l in range(4):
            g_ref[l] = (g_ref[l][0] + gi[l][0] / n, g_ref[l][1] + gi[l][1] / n)
            t_ref[l] = (t_ref[l][0] + mi[l][0] / n, t_ref[l][1] + mi[l][1] / n)
            t1_ref[l] = (t1_ref[l][0] + mi[l][2] / n, t1_ref[l][1] + mi[l][3] / n)
    assert float(stats[0]) / (n * W * H) == pytest.approx(loss_ref, rel=1e-2)
    worst = []
    for l in range(4):
        for a, b, t, t1 in zip(g_gpu[l], g_ref[l], t_ref[l], t1_ref[l]):
            bound = 2.0 ** -6 * np.abs(b) + 2.0 ** -8 * t + 2.0 ** -14 * t1
            bad = np.abs(a - b) > bound
            worst.append(float(np.max(np.abs(a - b) / np.maximum(bound, 1e-30))))
            assert not bad.any(), (l, np.argwhere(bad)[:5].tolist(), a[bad][:5], b[bad][:5], t[bad][:5])
    print("gradient elements, worst |gpu - oracle| / bound per layer (weights, bias):",
          " ".join(f"{w:.3g}" for w in worst))


def test_training_reduces_loss(slic_gpu):
    import torch
    from paper_1509_04232_gb300.warmstart import WarmStartNet, training_batch
    net = WarmStartNet(256, 256, 16, max_batch=8, seed=1)
    imgs, slots = training_batch(net, 0, 8, torch.device("cuda"))
    stats = torch.zeros(2, dtype=torch.float32, device="cuda")
    losses = []
    for step in range(60):
        net.train_step(imgs, slots, 3e-3, stats)
        losses.append(float(stats[0].item()) / (8 * 256 * 256))
    assert losses[-1] < 0.7 * losses[0], losses[::10]


def test_training_targets_agree_with_oracle(slic_gpu):
    """The GPU full-iteration labels used as training targets agree with the
    FP64 oracle's (before connectivity)."""
    import torch
    from paper_1509_04232_gb300.warmstart import reference_labels
    host = np.stack([synth.train_image(i) for i in range(3)])
    got = reference_labels(torch.from_numpy(host).cuda()).cpu().numpy()
    for i in range(3):
        ref = oracle.slic(host[i], S=16, m=10.0, iterations=10, enforce_connectivity=False)
        assert np.mean(got[i] == ref["labels_pre"]) >= 0.995


def test_trained_network_beats_grid_start_at_equal_iterations(slic_gpu, tmp_path):
    """Ablation: after a short training run, starting from the network's
    labels and doing one assignment agrees better with the full-iteration
    result than starting from the grid and doing one assignment; the gain is
    reported. A checkpoint round trip reproduces the same labels."""
    import torch
    from paper_1509_04232_gb300 import warmstart as ws
    net = ws.WarmStartNet(256, 256, 16, max_batch=64, seed=2)
    ws.train(net, n_images=4096, batch=64, epochs=2, lr=2e-3, first_image=0)
    imgs = torch.from_numpy(np.stack([synth.train_image(50_000 + i) for i in range(16)])).cuda()
    ref, _ = ws.plain_segment(imgs, 10)
    grid1, _ = ws.plain_segment(imgs, 0)
    warm1, _ = ws.warm_start_segment(net, imgs, 0)
    a_grid, a_warm = ws.agreement(grid1, ref), ws.agreement(warm1, ref)
    print(f"agreement with 10 iterations after one assignment: grid start {a_grid:.4f}, "
          f"network start {a_warm:.4f} (gain {a_warm - a_grid:+.4f})")
    assert a_warm > a_grid + 0.02
    path = str(tmp_path / "net.npz")
    net.save(path)
    net2 = ws.WarmStartNet(256, 256, 16, max_batch=16, seed=99)
    net2.load(path)
    l1 = torch.empty((16, 256, 256), dtype=torch.int32, device="cuda")
    l2 = torch.empty_like(l1)
    net.forward(imgs, labels=l1)
    net2.forward(imgs, labels=l2)
    assert torch.equal(l1, l2)


@pytest.mark.parametrize("W,H,n", [(1920, 48, 2), (1000, 41, 3)])
def test_forward_several_tiles_per_cta(slic_gpu, W, H, n):
    """Enough 120-pixel tiles that every persistent CTA takes several, so the
    input-stage ring and both accumulator buffers are reused (1536 and 1080
    tiles over the 2-CTA-per-SM grid); the second size has a ragged last
    tile. Logits of the whole batch against the oracle, and the fused
    labels-only path against the oracle's argmax."""
    import torch
    S = 16
    net, host, imgs = _setup(slic_gpu, n=n, W=W, H=H, S=S, seed=11)
    logits = torch.empty((n, H, W, 16), dtype=torch.float32, device="cuda")
    labels = torch.empty((n, H, W), dtype=torch.int32, device="cuda")
    net.forward(imgs, logits=logits)
    net.forward(imgs, labels=labels)
    torch.cuda.synchronize()
    net.status()
    params = _split(net.params())
    valid = NO.slot_mask(H, W, S)
    for i in range(n):
        ref, _ = NO.forward(_oracle_input(host[i], S), params, bf16=True)
        scale = max(1.0, np.abs(ref).max())
        got = logits[i].cpu().numpy()
        assert np.max(np.abs(got[..., :9] - ref)) <= 2e-2 * scale
        z = np.where(valid, ref, -np.inf)
        top2 = np.sort(z, axis=-1)[..., -2:]
        clear = (top2[..., 1] - top2[..., 0]) > 2e-2 * scale
        want = NO.labels_from_slots(np.argmax(z, axis=-1), S)
        assert np.all((labels[i].cpu().numpy() == want) | ~clear)


def test_forward_full_hd_batch_sampled(slic_gpu):
    """The bench's network launch configuration: 8 frames of 1920x1080,
    S=16 (three of them checked). The oracle evaluates sampled pixels one by
    one on the 9x9 window
    that determines them (four 3x3 layers), cut from its input channels of
    the whole frame and clipped at the image border, where every layer's zero
    padding then falls as on the device."""
    import torch
    W, H, S, n = 1920, 1080, 16, 8
    from paper_1509_04232_gb300.warmstart import WarmStartNet
    net = WarmStartNet(W, H, S, max_batch=n, seed=7)
    host = np.stack([synth.hd_image(40 + i, W, H) for i in range(n)])
    imgs = torch.from_numpy(host).cuda()
    logits = torch.empty((n, H, W, 16), dtype=torch.float32, device="cuda")
    labels = torch.empty((n, H, W), dtype=torch.int32, device="cuda")
    net.forward(imgs, logits=logits)
    net.forward(imgs, labels=labels)
    torch.cuda.synchronize()
    net.status()
    params = _split(net.params())
    rng = np.random.default_rng(5)
    ns_c, ns_r = -(-W // S), -(-H // S)
    fixed = [(0, 0), (0, W - 1), (H - 1, 0), (H - 1, W - 1), (1, 119), (2, 120), (540, 239), (541, 240),
             (H - 2, 1799), (H - 1, 1800), (7, W - 2), (H // 2, 1)]
    for i in (0, 4, 7):  # the oracle's input channels take seconds per 1080p frame
        x0 = _oracle_input(host[i], S)
        pts = fixed + [(int(rng.integers(0, H)), int(rng.integers(0, W))) for _ in range(36)]
        got_l = logits[i].cpu().numpy()
        got_lab = labels[i].cpu().numpy()
        for y, x in pts:
            r0, r1, c0, c1 = max(0, y - 4), min(H, y + 5), max(0, x - 4), min(W, x + 5)
            ref_win, _ = NO.forward(x0[r0:r1, c0:c1], params, bf16=True)
            ref = ref_win[y - r0, x - c0]
            scale = max(1.0, np.abs(ref).max())
            assert np.max(np.abs(got_l[y, x, :9] - ref)) <= 2e-2 * scale, (i, y, x)
            cx, cy = x // S, y // S
            ok = [0 <= cx + t % 3 - 1 < ns_c and 0 <= cy + t // 3 - 1 < ns_r for t in range(9)]
            z = np.where(ok, ref, -np.inf)
            top2 = np.sort(z)[-2:]
            if top2[1] - top2[0] > 2e-2 * scale:
                t = int(np.argmax(z))
                assert got_lab[y, x] == (cy + t // 3 - 1) * ns_c + cx + t % 3 - 1, (i, y, x)

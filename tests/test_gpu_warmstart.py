"""The learned warm start behind the C ABI (slic_batch_set_warmstart,
slic_set_warmstart) against an oracle chain: the GPU network's labels are
handed to the FP64 oracle, whose update turns them into member-mean centres
(Sec. 3 "Updating the cluster center") and whose whole run continues from
those centres (oracle.slic with init_centres). Tolerances as in the parity
tests: initial centres within 1e-4 max(1, |ref|) with exact counts, whole
runs at >= 99.5 % label agreement; the batched and the single-frame calls
are bit-identical."""
import numpy as np
import pytest

import oracle
from paper_1509_04232_gb300 import synth

pytestmark = pytest.mark.gpu

AGREE_MIN = 0.995
CENTRE_TOL = 1e-4


def _frames(n, W, H, seed0, regions=40, sigma=8.0):
    return np.stack([synth.voronoi_frame(W, H, regions, sigma, seed0 + i) for i in range(n)])


def _net_labels(net, imgs):
    import torch
    out = torch.empty(imgs.shape[:3], dtype=torch.int32, device="cuda")
    for b0 in range(0, imgs.shape[0], net.max_batch):
        net.forward(imgs[b0:b0 + net.max_batch], labels=out[b0:b0 + net.max_batch])
    torch.cuda.synchronize()
    net.status()
    return out.cpu().numpy()


def _oracle_chain(img, net_labels, S, m, iterations):
    feat = oracle.convert(img)
    init = oracle.update(feat, net_labels, oracle.init_centres(feat, S))
    return init, oracle.slic(img, S=S, m=m, iterations=iterations, init_centres=init)


@pytest.mark.parametrize("W,H,S,iterations,n,max_batch", [
    (320, 240, 16, 0, 3, 2),     # net + one assignment; three frames, forward in chunks of two
    (320, 240, 16, 3, 3, 4),
    (333, 257, 13, 2, 2, 2),     # ragged grid (partial last cells), S not a multiple of 4
])
def test_batch_warm_start_matches_oracle_chain(slic_gpu, W, H, S, iterations, n, max_batch):
    import torch
    from paper_1509_04232_gb300.warmstart import WarmStartNet
    pkg = slic_gpu
    m = 10.0
    host = _frames(n, W, H, 700 + W + iterations)
    imgs = torch.from_numpy(host).cuda()
    net = WarmStartNet(W, H, S, max_batch=max_batch, seed=5 + iterations)
    bs = pkg.BatchSegmenter([dict(width=W, height=H, S=S, m=m)] * n, iterations=iterations)
    bs.bind([imgs[i] for i in range(n)])
    bs.set_warmstart(net)
    labels, centres = bs.segment()
    torch.cuda.synchronize()
    bs.status()
    nl = _net_labels(net, imgs)
    for i in range(n):
        init, ref = _oracle_chain(host[i], nl[i], S, m, iterations)
        got = labels[i].cpu().numpy()
        agree = float(np.mean(got == ref["labels"]))
        assert agree >= AGREE_MIN, (i, agree)
        if iterations == 0:
            # the returned centres are the ones the labels were assigned
            # against: the member means of the network's labels
            c = centres[i].cpu().numpy()
            assert np.array_equal(c[:, 5], init[:, 5])
            assert np.all(np.abs(c[:, :5] - init[:, :5]) <= CENTRE_TOL * np.maximum(1.0, np.abs(init[:, :5])))


def test_warm_start_full_hd_sampled_frame(slic_gpu):
    """The bench's learned launch configuration (32 frames of 1920x1080,
    S=16, m=10) with one frame checked against the oracle chain."""
    import torch
    from paper_1509_04232_gb300 import warmstart as ws
    W, H, S, n, it = 1920, 1080, 16, 32, 1
    host = np.stack([synth.hd_image(500 + i, W, H) for i in range(n)])
    imgs = torch.from_numpy(host).cuda()
    net = ws.WarmStartNet(W, H, S, max_batch=n, seed=3)
    labels, _ = ws.warm_start_segment(net, imgs, it)
    nl = _net_labels(net, imgs[5:6])
    _, ref = _oracle_chain(host[5], nl[0], S, 10.0, it)
    assert float(np.mean(labels[5].cpu().numpy() == ref["labels"])) >= AGREE_MIN


def test_warm_start_batch_equals_single_frame(slic_gpu):
    """Batched and single-frame warm starts give the same labels and centres
    bit for bit (4-channel input, 5 frames, forward chunks of 2)."""
    import torch
    from paper_1509_04232_gb300.warmstart import WarmStartNet
    pkg = slic_gpu
    W, H, S, n, it = 256, 192, 16, 5, 2
    host = _frames(n, W, H, 90)
    rgba = np.concatenate([host, np.full(host.shape[:3] + (1,), 255, np.uint8)], axis=-1)
    imgs = torch.from_numpy(np.ascontiguousarray(rgba)).cuda()
    net = WarmStartNet(W, H, S, max_batch=2, seed=1)
    bs = pkg.BatchSegmenter([dict(width=W, height=H, S=S, in_channels=4)] * n, iterations=it)
    bs.bind([imgs[i] for i in range(n)])
    bs.set_warmstart(net)
    bl, bc = bs.segment()
    seg = pkg.Segmenter(W, H, S=S, iterations=it, in_channels=4)
    seg.set_warmstart(net)
    for i in range(n):
        sl, sc = seg.segment(imgs[i])
        assert torch.equal(sl, bl[i]) and torch.equal(sc, bc[i]), i
    # disarming restores the plain path
    seg.set_warmstart(None)
    bs.set_warmstart(None)
    plain = pkg.Segmenter(W, H, S=S, iterations=it, in_channels=4)
    pl, pc = plain.segment(imgs[0])
    sl, sc = seg.segment(imgs[0])
    bl, bc = bs.segment()
    assert torch.equal(pl, sl) and torch.equal(pl, bl[0]) and torch.equal(pc, bc[0])


def test_warm_start_rejects_another_geometry(slic_gpu):
    from paper_1509_04232_gb300 import SlicError, SLIC_ERR_INVALID
    from paper_1509_04232_gb300.warmstart import WarmStartNet
    pkg = slic_gpu
    net = WarmStartNet(64, 48, 16, max_batch=1)
    for kw in (dict(width=64, height=48, S=8), dict(width=64, height=40, S=16), dict(width=64, height=48, S=16, m=20.0)):
        seg = pkg.Segmenter(kw["width"], kw["height"], S=kw["S"], m=kw.get("m", 10.0))
        with pytest.raises(SlicError) as ei:
            seg.set_warmstart(net)
        assert ei.value.status == SLIC_ERR_INVALID
        bs = pkg.BatchSegmenter([dict(kw)], iterations=1)
        with pytest.raises(SlicError) as ei:
            bs.set_warmstart(net)
        assert ei.value.status == SLIC_ERR_INVALID


def test_target_slots_from_the_library(slic_gpu):
    """slic_net_slots against the oracle's slot map, and labels outside the
    3x3 cell window flagged (slot 255, counted)."""
    import torch
    from oracle import net_oracle as NO
    from paper_1509_04232_gb300 import warmstart as ws
    W, H, S = 96, 72, 8
    host = _frames(2, W, H, 11)
    ref = [oracle.slic(host[i], S=S, m=10.0, iterations=4, enforce_connectivity=False)["labels_pre"] for i in range(2)]
    net = ws.WarmStartNet(W, H, S, max_batch=2)
    labels = torch.from_numpy(np.stack(ref)).cuda()
    slots = ws.target_slots(net, labels).cpu().numpy()
    for i in range(2):
        assert np.array_equal(slots[i], NO.slots_from_labels(ref[i], S).astype(np.uint8))
    bad = labels.clone()
    bad[0, 0, 0] = (H // S - 1) * (W // S) + W // S - 1   # the far corner's cell
    bad[1, 5, 5] = -1
    with pytest.raises(ValueError, match="2 labels outside"):
        ws.target_slots(net, bad)

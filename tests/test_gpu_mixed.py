"""The mixed-resolution batch at full size: 256 seeded frames (64 each of
640x480, 1280x720, 1920x1080 and 3840x2160; S from {8, 16, 32}, m from
{5, 10, 20}), 5 iterations, one launch per stage, in the autotuned launch
shape. Sampled frames (one per size) are checked against the oracle and bit
for bit against the single-frame path; every frame's labels are checked for
properties that hold at any size."""
import numpy as np
import pytest

import oracle
from paper_1509_04232_gb300 import synth

pytestmark = pytest.mark.gpu

SAMPLES = (0, 64, 128, 192)   # one frame of each size


def test_mixed_batch_full_size(slic_gpu, tmp_path):
    import torch
    pkg = slic_gpu
    specs = synth.mixed_batch_specs(256)
    frames = [dict(width=w, height=h, S=S, m=m) for (w, h, S, m) in specs]
    host = [synth.mixed_batch_frame(f, w, h) for f, (w, h, _, _) in enumerate(specs)]
    imgs = [torch.from_numpy(h).cuda() for h in host]
    bs = pkg.BatchSegmenter(frames, iterations=5)
    bs.bind(imgs)
    bs.autotune(str(tmp_path / "tune.jsonl"))
    labels, centres = bs.segment()
    torch.cuda.synchronize()
    bs.status()

    # every frame: labels are valid centre indices within three cells of the
    # pixel's own cell (the 3x3 window, widened by one cell per connectivity
    # pass: a pixel may adopt a neighbour's label)
    for f, (w, h, S, _) in enumerate(specs):
        lab = labels[f]
        ns_c, ns_r = -(-w // S), -(-h // S)
        assert int(lab.min()) >= 0 and int(lab.max()) < ns_c * ns_r
        ys = torch.arange(h, device=lab.device).view(h, 1) // S
        xs = torch.arange(w, device=lab.device).view(1, w) // S
        assert int((lab % ns_c - xs).abs().max()) <= 3
        assert int((lab // ns_c - ys).abs().max()) <= 3
        assert int((centres[f][:, 5] > 0).sum()) > 0

    for f in SAMPLES:
        w, h, S, m = specs[f]
        got = labels[f].cpu().numpy()
        ref = oracle.slic(host[f], S=S, m=m, iterations=5)
        assert np.mean(got == ref["labels"]) >= 0.995, f
        seg = pkg.Segmenter(w, h, S=S, m=m, iterations=5)
        l1, c1 = seg.segment(imgs[f])
        np.testing.assert_array_equal(got, l1.cpu().numpy())
        np.testing.assert_array_equal(centres[f].cpu().numpy(), c1.cpu().numpy())

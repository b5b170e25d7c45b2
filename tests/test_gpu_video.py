"""Video with the temporal warm start: every frame's labels against the FP64
oracle run with the same initialisation chain (its own previous-batch
centres); the grid mode against plain batched SLIC."""
import numpy as np
import pytest

import oracle
from paper_1509_04232_gb300 import synth

pytestmark = pytest.mark.gpu


def test_video_matches_oracle_chain(slic_gpu):
    import torch
    from paper_1509_04232_gb300.video import run_video
    T, W, H, batch = 12, 320, 240, 4
    host = np.stack([synth.video_frame(t, W, H) for t in range(T)])
    out = run_video(torch.from_numpy(host).cuda(), batch=batch, iterations=2, first_iterations=10)
    assert out["frames"] == T and len(out["agreement_vs_plain_10"]["per_frame"]) == T
    assert out["latency_ms"]["p99"] >= out["latency_ms"]["p50"] > 0
    # oracle with the same chain: first batch from the grid (10 it), later
    # batches from the previous batch's last frame's final centres (2 it)
    prev = None
    ref_labels = []
    for b in range(T // batch):
        its = 10 if prev is None else 2
        res = [oracle.slic(host[f], S=16, m=10.0, iterations=its, init_centres=prev)
               for f in range(b * batch, (b + 1) * batch)]
        prev = res[-1]["centres"]
        ref_labels += [r["labels"] for r in res]
    # and the GPU labels of the same run
    from paper_1509_04232_gb300 import BatchSegmenter
    gpu = []
    prev_t = None
    frames = torch.from_numpy(host).cuda()
    for b in range(T // batch):
        bs = BatchSegmenter([dict(width=W, height=H, S=16, m=10.0)] * batch,
                            iterations=10 if prev_t is None else 2)
        bs.bind([frames[f] for f in range(b * batch, (b + 1) * batch)],
                init_centres=[prev_t] * batch if prev_t is not None else None)
        labels, centres = bs.segment()
        prev_t = centres[-1].clone()
        gpu += [l.cpu().numpy() for l in labels]
    agree = [np.mean(g == r) for g, r in zip(gpu, ref_labels)]
    assert min(agree) >= 0.99, agree


def test_video_grid_mode_is_plain_slic(slic_gpu):
    """init="grid" segments every batch like plain batched SLIC; agreement
    and latency bookkeeping are consistent."""
    import torch
    from paper_1509_04232_gb300.video import run_video
    from paper_1509_04232_gb300.warmstart import agreement, plain_segment
    T, W, H = 8, 320, 240
    frames = torch.from_numpy(np.stack([synth.video_frame(t, W, H) for t in range(T)])).cuda()
    out = run_video(frames, batch=4, iterations=10, init="grid")
    assert out["agreement_vs_plain_10"]["min"] == 1.0          # 10 iterations from the grid = the reference
    out2 = run_video(frames, batch=4, iterations=2, init="grid")
    ref, _ = plain_segment(frames, 10)
    two, _ = plain_segment(frames, 2)
    assert abs(out2["agreement_vs_plain_10"]["mean"] - agreement(two, ref)) < 1e-9
    assert out2["frames_per_s"] > 0 and out2["latency_ms"]["p50"] > 0

"""Video stream: frames segmented in batches, every frame of a batch starting
from the final centres of the previous batch's last frame (the temporal warm
start), so a few iterations suffice; the first batch starts from the grid.

Run as ``python -m paper_1509_04232_gb300.video`` to print one JSON line
with frames/s, per-frame latency percentiles (batch completion minus batch
launch, inputs resident on the device) and the label agreement of every
frame with plain 10-iteration SLIC of the same frame.
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np


def run_video(frames, batch: int = 8, iterations: int = 2, S: int = 16, m: float = 10.0,
              reference_iterations: int = 10, first_iterations: int = 10, init: str = "previous", stream=None):
    """frames: uint8 CUDA tensor [T, H, W, 3] (device-resident).
    init="previous": the first batch starts from the grid with
    `first_iterations`, every later batch from the previous batch's last
    frame's final centres with `iterations` (temporal warm start).
    init="grid": every batch starts from the grid with `iterations`.
    Returns per-frame agreement with plain `reference_iterations` SLIC,
    batch latencies and throughput."""
    if init not in ("previous", "grid"):
        raise ValueError("init must be 'previous' or 'grid'")
    import torch
    from . import BatchSegmenter
    from .warmstart import agreement, plain_segment
    T, H, W, _ = frames.shape
    dev = frames.device
    stream = stream if stream is not None else torch.cuda.current_stream()
    n_batches = (T + batch - 1) // batch
    # one batch object per batch size (the last one may be short); centres of
    # the previous batch's last frame feed the next batch
    segs = {}
    prev = None
    labels_out = []
    lat_ms = []
    torch.cuda.synchronize()
    for b in range(n_batches):
        f0, f1 = b * batch, min(T, (b + 1) * batch)
        n = f1 - f0
        if init == "grid":
            prev = None
        key = (n, prev is None)
        if key not in segs:
            its = iterations if (prev is not None or init == "grid") else first_iterations
            segs[key] = BatchSegmenter([dict(width=W, height=H, S=S, m=m)] * n, iterations=its, device=dev)
        bs = segs[key]
        bs.bind([frames[i] for i in range(f0, f1)], init_centres=[prev] * n if prev is not None else None)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            labels, centres = bs.segment(stream)
            e1.record(stream)
            # next batch starts from this batch's last frame's final centres
            prev = centres[-1].clone() if init == "previous" else None
            labels_out += [l.clone() for l in labels]
        torch.cuda.synchronize()
        lat_ms += [e0.elapsed_time(e1)] * n
    total_ms = sum(lat_ms[f] for f in range(0, T, batch))
    # agreement with plain 10-iteration SLIC, frame by frame
    agree = []
    for f0 in range(0, T, batch):
        sub = frames[f0:f0 + batch]
        ref, _ = plain_segment(sub, reference_iterations, S, m)
        for i in range(sub.shape[0]):
            agree.append(agreement([labels_out[f0 + i]], [ref[i]]))
    for bs in segs.values():
        bs.status()
    return {"init": init, "frames": T, "batch": batch, "iterations": iterations,
            "first_batch_iterations": first_iterations if init == "previous" else iterations,
            "frames_per_s": T / (total_ms / 1e3),
            "latency_ms": {"p50": float(np.percentile(lat_ms, 50)), "p99": float(np.percentile(lat_ms, 99))},
            "agreement_vs_plain_10": {"mean": float(np.mean(agree)), "min": float(np.min(agree)),
                                      "per_frame": [round(a, 5) for a in agree]}}


def main(argv=None):
    import torch
    from . import build, synth
    ap = argparse.ArgumentParser(description="4K video with temporal warm start")
    ap.add_argument("--frames", type=int, default=120)
    ap.add_argument("--width", type=int, default=3840)
    ap.add_argument("--height", type=int, default=2160)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--iterations", type=int, default=2)
    args = ap.parse_args(argv)
    build.build_all()
    host = torch.empty((args.frames, args.height, args.width, 3), dtype=torch.uint8).pin_memory()
    for t in range(args.frames):
        host[t].numpy()[...] = synth.video_frame(t, args.width, args.height)
    frames = host.cuda()
    run_video(frames[: args.batch], args.batch, args.iterations)  # warm-up (module load, allocations)
    result = {"workload": f"{args.frames} frames {args.width}x{args.height}, 400 regions moving 0-4 px/frame, "
                          f"colour drift 2, noise 6; S=16, m=10; {args.batch} frames per launch"}
    for init in ("previous", "grid"):
        out = run_video(frames, args.batch, args.iterations, init=init)
        out["agreement_vs_plain_10"].pop("per_frame")
        result[init] = out
    print(json.dumps(result))
    return 0


if __name__ == "__main__":
    sys.exit(main())

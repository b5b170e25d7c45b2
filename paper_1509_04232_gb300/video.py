"""Video stream: frames segmented in batches, every frame of a batch starting
from the final centres of the previous batch's last frame (the temporal warm
start), so a few iterations suffice; the first batch starts from the grid.
Optionally the learned warm start is armed as well: the network's labels of
each frame, with the previous batch's centres for the cells the network
gives no pixel.

Run as ``python -m paper_1509_04232_gb300.video`` to print one JSON line
with frames/s, per-frame latency percentiles (batch completion minus batch
launch, inputs resident on the device), and per frame against plain
10-iteration SLIC of the same frame: the label agreement (label indices
must match), the achievable segmentation accuracy and the boundary recall
(both independent of how segments are numbered), and how far the chained
centres drift from their own cells.
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np


def segmentation_accuracy(labels, ref) -> float:
    """Achievable segmentation accuracy of `labels` against `ref` (int32 CUDA
    tensors [H, W]): every segment of `labels` takes the reference label it
    overlaps most, and the score is the fraction of pixels this gets right
    (1.0 for any renumbering of the reference)."""
    import torch
    a = labels.reshape(-1).to(torch.int64)
    b = ref.reshape(-1).to(torch.int64)
    key = a * (int(b.max().item()) + 1) + b
    pairs, counts = torch.unique(key, return_counts=True)
    seg = pairs // (int(b.max().item()) + 1)
    best = torch.zeros(int(a.max().item()) + 1, dtype=torch.int64, device=a.device)
    best.scatter_reduce_(0, seg, counts, reduce="amax")
    return float(best.sum().item()) / a.numel()


def boundary_recall(labels, ref, tol: int = 2) -> float:
    """Fraction of the reference's boundary pixels (a 4-neighbour with
    another label) that lie within `tol` pixels (Chebyshev) of a boundary
    pixel of `labels`."""
    import torch

    def edges(l):
        e = torch.zeros_like(l, dtype=torch.bool)
        e[:, 1:] |= l[:, 1:] != l[:, :-1]
        e[:, :-1] |= l[:, 1:] != l[:, :-1]
        e[1:, :] |= l[1:, :] != l[:-1, :]
        e[:-1, :] |= l[1:, :] != l[:-1, :]
        return e

    er, el = edges(ref), edges(labels).float()[None, None]
    near = torch.nn.functional.max_pool2d(el, 2 * tol + 1, stride=1, padding=tol)[0, 0] > 0
    n = int(er.sum().item())
    return float((er & near).sum().item()) / n if n else 1.0


def centre_drift(centres, W: int, H: int, S: int) -> float:
    """Largest distance (in units of S, Chebyshev) of a centre from the
    midpoint of the grid cell its label names; the 3x3 cell window of the
    assignment assumes it stays within about one cell."""
    import torch
    K = centres.shape[0]
    ns_c = -(-W // S)
    k = torch.arange(K, device=centres.device)
    cx, cy = k % ns_c, k // ns_c
    mx = (cx * S + torch.clamp((cx + 1) * S, max=W) - 1).float() / 2
    my = (cy * S + torch.clamp((cy + 1) * S, max=H) - 1).float() / 2
    live = centres[:, 5] > 0
    d = torch.maximum((centres[:, 3] - mx).abs(), (centres[:, 4] - my).abs())[live]
    return float(d.max().item()) / S if d.numel() else 0.0


def run_video(frames, batch: int = 8, iterations: int = 2, S: int = 16, m: float = 10.0,
              reference_iterations: int = 10, first_iterations: int = 10, init: str = "previous", stream=None,
              net=None):
    """frames: uint8 CUDA tensor [T, H, W, 3] (device-resident).
    init="previous": the first batch starts from the grid with
    `first_iterations`, every later batch from the previous batch's last
    frame's final centres with `iterations` (temporal warm start).
    init="grid": every batch starts from the grid with `iterations`.
    net: a network (warmstart.WarmStartNet for this geometry) armed as the
    learned warm start of every batch after the first (its labels' member
    means, the previous centres where it gives a cell no pixel).
    Returns per-frame agreement, segmentation accuracy and boundary recall
    against plain `reference_iterations` SLIC, the centre drift, batch
    latencies and throughput."""
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
    drift = []
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
            if net is not None and prev is not None:
                segs[key].set_warmstart(net)
        bs = segs[key]
        bs.bind([frames[i] for i in range(f0, f1)], init_centres=[prev] * n if prev is not None else None,
                stream=stream)
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
        drift.append(max(centre_drift(c, W, H, S) for c in centres))
    total_ms = sum(lat_ms[f] for f in range(0, T, batch))
    # against plain 10-iteration SLIC, frame by frame
    agree, asa, br = [], [], []
    for f0 in range(0, T, batch):
        sub = frames[f0:f0 + batch]
        ref, _ = plain_segment(sub, reference_iterations, S, m)
        for i in range(sub.shape[0]):
            agree.append(agreement([labels_out[f0 + i]], [ref[i]]))
            asa.append(segmentation_accuracy(labels_out[f0 + i], ref[i]))
            br.append(boundary_recall(labels_out[f0 + i], ref[i]))
    for bs in segs.values():
        bs.status()
    return {"init": init + ("+learned" if net is not None else ""), "frames": T, "batch": batch,
            "iterations": iterations,
            "first_batch_iterations": first_iterations if init == "previous" else iterations,
            "frames_per_s": T / (total_ms / 1e3),
            "latency_ms": {"p50": float(np.percentile(lat_ms, 50)), "p99": float(np.percentile(lat_ms, 99))},
            "agreement_vs_plain_10": {"mean": float(np.mean(agree)), "min": float(np.min(agree)),
                                      "per_frame": [round(a, 5) for a in agree]},
            "segmentation_accuracy_vs_plain_10": {"mean": float(np.mean(asa)), "min": float(np.min(asa))},
            "boundary_recall_vs_plain_10": {"mean": float(np.mean(br)), "min": float(np.min(br)), "tolerance_px": 2},
            "centre_drift_cells": {"max": float(np.max(drift)), "last_batch": drift[-1]}}


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

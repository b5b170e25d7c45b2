"""Benchmark: 1080p SLIC frames/s at >= 99 % label agreement, on GB300.

The metric compares the batched plain path with the batched learned warm
start at equal quality: each runs at the smallest iteration count whose
mean label agreement with 10-iteration SLIC (connectivity on for both)
reaches 99 % on an evaluation set of 64 seeded synthetic 1920x1080 frames
(400 Voronoi regions, noise 6; S=16, m=10), and `value` is the faster of the
two. One step is one batch of 32 such frames (the throughput frames, other
seeds), one CUDA graph (one batched launch per stage) at that iteration
count; the batch's inputs (32 x 6.2 MB of RGB, 32 x 8.3 MB of labels) are
larger than the 129 MB L2, so no flush is needed between steps.

Prints ONE JSON line (rank 0). Keys beyond the base contract:
  quality       the agreement-vs-iterations curves of both methods, their
                iteration counts at 99 % and frames/s there, the network's
                training and its forward against the bf16 tensor roofline
  roofline      the dominant kernel (the pipelined assignment pass) against
                its bound (the square-root pipe), with its HBM view
  cpu_baseline  the FP64 CPU oracle timed on a bounded sample over all host
                cores (one process per core), with a one-core figure beside it
  e2e           the same metric through the public API with host buffers
  gpu_launches  kernel launches of this library inside the timed region
  clocks        SM clocks sampled by nvidia-smi during the timed region
  throughput_5_iterations  plain batched SLIC at 5 iterations (32 x 1080p)
  single_frame  graph-captured slic_segment latency: 1920x1080 S=16 and
                640x480 K=1200, 5 iterations
  sec2_options  the stopping test with early exit, the seed perturbation,
                input variants and component connectivity
  mixed_batch   the 256-frame mixed-resolution batch
  video         120 frames of 3840x2160 with the temporal warm start

``--impl reference`` times the FP64 CPU oracle itself (the only reference
implementation of the method in this repository) on the same frames at 10
iterations.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

W, H, S, M = 1920, 1080, 16, 10.0
ITERS = 5          # the plain throughput configuration: 32 frames 1920x1080, 5 iterations
FULL_ITERS = 10    # the full-iteration result the agreement bar refers to
EVAL_FRAMES = 64   # the evaluation set of the agreement bar
AGREE_BAR = 0.99
METRIC = "1080p SLIC frames/s (batched+learned vs plain GPU) at \u226599% label agreement"
UNIT = "frames/s"


# --- multi-process helpers (also exercised by the CPU tests with gloo) -------

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def frame_seeds(batch: int, rank: int) -> list[int]:
    """Each rank segments its own batch of distinct frames (weak scaling)."""
    return [rank * batch + f for f in range(batch)]


def max_over_ranks(value: float, world: int, device=None) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int, device=None):
    if world <= 1:
        return
    import torch.distributed as dist
    if device is not None and dist.get_backend() == "nccl":
        dist.barrier(device_ids=[device.index])
    else:
        dist.barrier()


# --- clocks -----------------------------------------------------------------

class ClockSampler:
    """nvidia-smi sampler of SM clocks and throttle reasons (read-only)."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9 and f[1].replace(".", "").isdigit():
                    rows.append(f)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


# --- peaks ------------------------------------------------------------------

def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# --- the CPU oracle legs ----------------------------------------------------

def _oracle_frame(job):
    """One oracle run on a 1080p frame (in a spawned worker process)."""
    import oracle
    img, iterations = job
    oracle.slic(img, S=S, m=M, iterations=iterations, enforce_connectivity=True)
    return 0


def _oracle_ready(_):
    import oracle
    oracle.build()
    return os.getpid()


def oracle_frames_per_s(frames, procs: int, iterations: int) -> float:
    """Wall-clock frames/s of the FP64 oracle (as it stands) over `frames`,
    one frame per task on `procs` spawned worker processes (spawn, not fork:
    the parent may hold a CUDA context)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        pool.map(_oracle_ready, range(procs))  # workers up and the library loaded, untimed
        t0 = time.perf_counter()
        pool.map(_oracle_frame, [(f, iterations) for f in frames], chunksize=1)
        dt = time.perf_counter() - t0
    return len(frames) / dt


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_1509_04232_gb300 import synth
    oracle.build()
    procs = host_cores()
    # inputs are generated before timing, as on the GPU side; one step = one
    # frame, the steps spread over all host cores
    warm = [synth.hd_image(19_000 + k, W, H) for k in range(args.warmup)]
    frames = [synth.hd_image(20_000 + k, W, H) for k in range(args.steps)]
    oracle_frames_per_s(warm, procs, FULL_ITERS)
    value = oracle_frames_per_s(frames, procs, FULL_ITERS)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "1 frame 1920x1080 per step, S=16 m=10, 10 it (the agreement "
                                                        "reference), connectivity",
                                            "global_batch": 1, "iterations": FULL_ITERS,
                                            "parallelism": f"{procs} host processes, one frame each at a time"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                             "sample": f"{args.steps} frames 1920x1080 over {procs} processes"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# --- the GPU path -----------------------------------------------------------

def _plain_batch(pkg, images, iterations, dev, tuning=None, **kw):
    """A bound batch of the throughput frames (plain path)."""
    bs = pkg.BatchSegmenter([dict(width=W, height=H, S=S, m=M)] * len(images), iterations=iterations, device=dev, **kw)
    bs.bind(list(images))
    if tuning:
        bs.set_tuning(*tuning)
    return bs


def _capture(fn, stream):
    """One eager call (module loading, first-use set-up), then a CUDA graph of it."""
    import torch
    with torch.cuda.stream(stream):
        fn()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        fn()
    torch.cuda.synchronize()
    return g


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_1509_04232_gb300 as pkg
    from paper_1509_04232_gb300 import build, synth
    build.build_all()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count

    if args.train_only:  # the warm-start network's training alone (a profiling command)
        from paper_1509_04232_gb300 import warmstart as ws
        net = ws.WarmStartNet(256, 256, S, max_batch=64, seed=0, m=M)
        t0 = time.time()
        hist = ws.train(net, n_images=args.train_images, batch=64, epochs=1, lr=2e-3, log_every=50)
        torch.cuda.synchronize()
        net.status()
        if rank == 0:
            print(json.dumps({"training": {"images": args.train_images, "seconds": time.time() - t0,
                                           "final_loss": hist[-1][1] if hist else None}}))
        net.close()
        return 0
    if args.mixed_only:  # the mixed batch alone (a profiling command)
        stream = torch.cuda.Stream(device=dev)
        if rank == 0:
            print(json.dumps({"mixed_batch": mixed_batch_throughput(args, pkg, stream, dev)}))
        return 0
    if args.components_only:  # component connectivity on the bench frames (a profiling command)
        stream = torch.cuda.Stream(device=dev)
        if rank == 0:
            print(json.dumps({"component_connectivity": components_step(args, pkg, stream, dev)}))
        return 0

    B = args.batch
    seeds = frame_seeds(B, rank)
    host = torch.empty((B, H, W, 3), dtype=torch.uint8).pin_memory()
    for i, sd in enumerate(seeds):
        synth.voronoi_frame(W, H, 400, 6.0, synth.seed_of(1, sd), out=host[i].numpy())
    images = host.to(dev)
    frames = [images[f] for f in range(B)]
    stream = torch.cuda.Stream(device=dev)
    tune_cache = os.path.join(tempfile.gettempdir(), "slicgb_autotune.jsonl")

    # --- the agreement bar: iteration sweeps of both methods on the eval set ---
    if args.iterations is not None:  # a fixed count (profiling commands): no sweep, no learned leg
        quality, net_small = {"plain_iterations_at_99": args.iterations, "sweep": "skipped (--iterations)"}, None
    else:
        quality, net_small = agreement_sweeps(args, pkg, dev, stream)
    n_plain = quality["plain_iterations_at_99"]
    n_learned = quality.get("learned_iterations_at_99")

    # --- the plain path at its iteration count, autotuned, one graph per step ---
    bs = _plain_batch(pkg, frames, n_plain, dev)
    if args.tuning:  # a fixed launch shape (profiling commands): no autotuning
        tuning = (tuple(int(v) for v in args.tuning.split(",")) + (0, 1))[:6]
        bs.set_tuning(*tuning)
    else:
        tuning = bs.autotune(tune_cache, stream=stream)
    ctas_per_sm, stages, rows, tile_h, fused, groups = tuning
    K_EFF = bs.K_eff[0]
    n0 = bs.info[1]
    graph = _capture(lambda: bs.segment(stream=stream), stream)
    launches_per_step = (bs.info[1] - n0) // 2
    plain_ms = _graph_ms(graph, stream, args, world, dev)
    method = {"name": "plain", "iterations": n_plain, "frames_per_s": world * B / (plain_ms / 1e3)}
    learned_fps = None
    if n_learned is not None and net_small is not None:
        from paper_1509_04232_gb300 import warmstart as ws
        net = ws.WarmStartNet(W, H, S, max_batch=B, seed=0, m=M)
        net.set_params(net_small.params())
        pipe = ws.WarmStartPipeline(net, frames, n_learned, m=M)
        g_l = _capture(lambda: pipe.run(stream), stream)
        learned_fps = world * B / (_graph_ms(g_l, stream, args, world, dev) / 1e3)
        quality["learned_frames_per_s_at_99"] = learned_fps
        if learned_fps > method["frames_per_s"]:
            method = {"name": "learned", "iterations": n_learned, "frames_per_s": learned_fps}
            graph, bs, launches_per_step = g_l, pipe.bs, None
    quality["plain_frames_per_s_at_99"] = world * B / (plain_ms / 1e3)
    quality["headline_method"] = method["name"]

    # --- device-resident throughput of the headline method ---
    clocks = ClockSampler(local)
    clocks.start()
    with torch.cuda.stream(stream):  # replay() launches on the current stream
        for _ in range(args.warmup):
            graph.replay()
        torch.cuda.synchronize()
        barrier(world, dev)
        torch.cuda.synchronize()
        # an event after every replay gives the per-step distribution too
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        evs[0].record(stream)
        for k in range(args.steps):
            graph.replay()
            evs[k + 1].record(stream)
    torch.cuda.synchronize()
    barrier(world, dev)
    torch.cuda.synchronize()
    clock_info = clocks.stop()
    ms = max_over_ranks(evs[0].elapsed_time(evs[-1]), world, dev) / args.steps
    step_ms = np.array([evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)])
    value = world * B / (ms / 1e3)
    if launches_per_step is None:
        launches_per_step = 0  # (the learned step: counted below)

    # --- dominant kernel: event-timed replays of the plain step ---
    # Each replay records one event pair per assignment launch. One launch
    # per pass: pass order 0..n, and passes 1..n-1 run the dominant kernel
    # (the pipelined middle pass, k_assign_pipe<0,1,MINB,ROWS,TILE_H>: MINB
    # = 2 for 32x64 tiles, 4 for the 32x32 two-row-group build and for the
    # one-row 64-register build the autotuner picks at 4 CTAs per SM, else
    # 3). Fused passes: the fused launch (passes 0..n-1 with their updates,
    # k_assign_multi<1,MINB,ROWS,TILE_H>) and the last pass; the fused launch
    # is the dominant kernel, with n passes' work. With the timers on, the
    # batch runs as one group of frames (concurrent groups would share the
    # GPU during a launch, so its duration would not be its own).
    pb = bs if method["name"] == "plain" else _plain_batch(pkg, frames, n_plain, dev, tuning)
    # The kernel on its own: one group of frames at full occupancy in the
    # tuned tile shape, stages and rows (the step itself runs its groups
    # concurrently, each launch sharing the GPU with the others').
    pb.set_tuning(0, stages, rows, tile_h, fused=fused, groups=1)
    occ_alone = pb.info[2]
    pkg.slic_batch_profile_enable(pb.handle, True)
    graph_prof = _capture(lambda: pb.segment(stream=stream), stream)
    pkg.slic_batch_profile_enable(pb.handle, False)
    minb = 2 if tile_h == 64 else (4 if (rows == 2 or occ_alone >= 4) else 3)
    fused_dom = bool(fused) and n_plain >= 1
    kname = (f"k_assign_multi<1,{minb},{rows},{tile_h}>" if fused_dom else
             f"k_assign_pipe<0,1,{minb},{rows},{tile_h}>")
    passes_per_launch = n_plain if fused_dom else 1
    mid = []
    for _ in range(max(3, min(args.steps, 10))):
        with torch.cuda.stream(stream):
            graph_prof.replay()
        torch.cuda.synchronize()
        t = pkg.slic_batch_profile_times(pb.handle)
        if fused_dom:
            mid.append(t[-2])  # this replay's fused launch
        else:
            t = t[-(n_plain + 1):]  # this replay's passes
            mid += [t[p] for p in (range(1, n_plain) if n_plain >= 2 else range(n_plain + 1))]
    mid_ms = float(np.mean(mid))
    N = W * H
    # Algorithmic work of one middle-pass launch (all B frames): 12 bytes of
    # features read per pixel (centre windows and sums are < 1%), 18 square
    # roots per pixel (2 for each of the 9 candidates of Eq. 1); a fused
    # launch does that for each of its passes.
    bytes_per_launch = B * N * 12 * passes_per_launch
    achieved_gbs = bytes_per_launch / (mid_ms / 1e3) / 1e9
    sqrt_per_launch = B * N * 18 * passes_per_launch
    peaks, peak_kind = measured_peaks()
    sm_max = clock_info.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    xu_peak = 16 * sms * sm_max * 1e6 / 1e12
    achieved_tops = sqrt_per_launch / (mid_ms / 1e3) / 1e12
    # In the step as timed: the square roots of all its assignment passes
    # over the whole step time (conversion, updates and connectivity
    # included, so a lower bound on the rate the passes ran at).
    in_step_tops = B * N * 18 * (n_plain + 1) / (ms / 1e3) / 1e12 if method["name"] == "plain" else None
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "assign_traffic.txt")
    if os.path.exists(tfile):
        # "kernel <name>" and "dram_bytes_per_frame <n>" lines, from one ncu
        # capture of the current kernel (removed whenever the kernel changes)
        kv = dict(line.split(None, 1) for line in open(tfile) if line.strip() and not line.startswith("#"))
        if kv.get("kernel", "").strip() == kname:
            traffic = float(kv["dram_bytes_per_frame"]) * B * passes_per_launch

    # --- end to end through the C ABI with host buffers ---
    # slic_batch_segment_host: H2D copy of the step's frames, the step, D2H
    # copy of labels and centres. Two batches bound to separate device
    # buffers alternate on two streams, so one step's copies overlap the
    # other's kernels; every step still moves all of its own bytes. With
    # frame groups each group's stream copies its own frames in and out, so
    # more groups overlap more of the copies: the leg takes the faster of the
    # tuned grouping and 4 groups in a short trial, then times the steps.
    h2d = B * H * W * 3
    d2h = B * H * W * 4 + B * K_EFF * 6 * 4
    e_iters = method["iterations"]
    h_imgs = [host[f] for f in range(B)]

    def e2e_run(e_groups, steps, warm):
        pair = []
        for _ in range(2):
            eb = pkg.BatchSegmenter([dict(width=W, height=H, S=S, m=M)] * B, iterations=e_iters, device=dev)
            eb.dimg = torch.empty_like(images)  # one allocation: the step's frames move with one copy
            eb.bind([eb.dimg[f] for f in range(B)])
            eb.set_tuning(ctas_per_sm, stages, rows, tile_h, fused=fused, groups=e_groups)
            if method["name"] == "learned":
                eb.set_warmstart(net)
            pair.append((eb, torch.cuda.Stream(device=dev), torch.empty((B, H, W), dtype=torch.int32).pin_memory(),
                         torch.empty((B, K_EFF, 6), dtype=torch.float32).pin_memory()))

        def host_step(k):
            b_, s_, hl, hc = pair[k & 1]
            b_.segment_host(h_imgs, [hl[f] for f in range(B)], [hc[f] for f in range(B)], stream=s_)

        for k in range(warm):
            host_step(k)
        torch.cuda.synchronize()
        barrier(world, dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(pair[0][1])
        pair[1][1].wait_event(e0)
        n_before = sum(p_[0].info[1] for p_ in pair)
        for k in range(steps):
            host_step(k)
        join = torch.cuda.Event()
        join.record(pair[1][1])
        pair[0][1].wait_event(join)
        e1.record(pair[0][1])
        torch.cuda.synchronize()
        ms_ = max_over_ranks(e0.elapsed_time(e1), world, dev) / steps
        launches = (sum(p_[0].info[1] for p_ in pair) - n_before) // steps
        for p_ in pair:
            p_[0].close()
        return ms_, launches

    e_groups = groups
    alt = min(4, B)
    if method["name"] == "plain" and alt != groups:
        trial = {g_: e2e_run(g_, 5, 3)[0] for g_ in (groups, alt)}
        e_groups = min(trial, key=trial.get)
    e2e_ms, e2e_launches = e2e_run(e_groups, args.steps, args.warmup)
    e2e_value = world * B / (e2e_ms / 1e3)
    if launches_per_step == 0:
        launches_per_step = e2e_launches

    # --- context: plain throughput at 5 iterations ---
    b5 = _plain_batch(pkg, frames, ITERS, dev, tuning)
    g5 = _capture(lambda: b5.segment(stream=stream), stream)
    ms5 = _graph_ms(g5, stream, args, world, dev)
    thr5 = {"iterations": ITERS, "frames_per_s": world * B / (ms5 / 1e3), "ms_per_step": ms5,
            "megapixels_per_s": world * B * N / 1e6 / (ms5 / 1e3),
            "agreement_with_10_iterations": quality.get("plain_agreement_by_iterations", {}).get(str(ITERS))}
    b5.close()

    single = None if args.no_single else single_frame_latency(args, pkg, stream, dev, images[0])
    mixed = None
    if rank == 0 and not args.no_mixed:
        mixed = mixed_batch_throughput(args, pkg, stream, dev)
    options = None
    if not args.no_options:
        options = sec2_options(args, pkg, images, B, stream, world, dev, tuning)
    video = None
    if rank == 0 and not args.no_video:
        video = video_context(args, pkg, dev, net_small)

    # --- CPU baseline: the FP64 oracle on a bounded sample (rank 0, N=1) ---
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        procs = host_cores()
        n_cpu = args.cpu_frames or 2 * procs
        sample = [synth.hd_image(10_000 + i, W, H) for i in range(n_cpu)]
        fps = oracle_frames_per_s(sample, procs, e_iters)
        fps1 = oracle_frames_per_s(sample[:2], 1, e_iters)
        cpu = {"value": fps, "unit": UNIT, "cores": procs, "kind": "oracle",
               "sample": f"{n_cpu} frames 1920x1080 (S=16, m=10, {e_iters} iterations, connectivity) over {procs} "
                         f"processes",
               "single_core": {"value": fps1, "sample": "2 of those frames on 1 process"}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms,
            "step_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{B}x1080p/step, S=16 m=10, {method['name']} at {method['iterations']} it "
                                   f"(>=99% agreement with 10 it)",
                       "method": method["name"], "iterations": method["iterations"],
                       "global_batch": world * B, "frames_per_gpu": B, "megapixels_per_s": value * N / 1e6,
                       "parallelism": f"replicas x{world} (frames sharded, no collective)",
                       "l2": "inputs larger than L2 (B x 6.2 MB RGB + B x 8.3 MB labels per step)",
                       "graph": "one CUDA graph per step (one batched launch per stage)",
                       "ctas_per_sm": ctas_per_sm, "pipeline_stages": stages, "row_groups_per_warp": rows,
                       "tile": f"32x{tile_h}", "fused_passes": bool(fused), "frame_groups": groups},
            "roofline": {"kernel": (f"{kname} (passes 0..{n_plain - 1} with their updates, all frames)" if fused_dom
                                    else f"{kname} (middle assignment pass, all frames)"), "bound": "alu",
                         "unit": "Tsqrt/s", "achieved": achieved_tops, "peak": xu_peak, "frac": achieved_tops / xu_peak,
                         "peak_source": f"16 MUFU lanes/clk/SM x {sms} SMs x max SM clock (recipe unit counts)",
                         "traffic": traffic, "avg_launch_us": mid_ms * 1e3, "launches_timed": len(mid),
                         "measured_as": f"one frame group at full occupancy ({occ_alone} CTAs/SM); the step runs "
                                        f"{groups} group(s) concurrently at {ctas_per_sm} CTAs/SM each",
                         "in_step": {"achieved": in_step_tops,
                                     "frac": in_step_tops / xu_peak if in_step_tops else None,
                                     "what": "all assignment passes' square roots / step time"},
                         "hbm": {"achieved": achieved_gbs, "peak": peaks["hbm_gbs"],
                                 "frac": achieved_gbs / peaks["hbm_gbs"], "unit": "GB/s",
                                 "peak_kind": peak_kind, "algorithmic_bytes_per_launch": bytes_per_launch}},
            "cpu_baseline": cpu,
            "quality": quality,
            "throughput_5_iterations": thr5,
            "single_frame": single,
            "sec2_options": options,
            "mixed_batch": mixed,
            "video": video,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "frame_groups": e_groups},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clock_info,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def single_frame_latency(args, pkg, stream, dev, image):
    """slic_segment on one frame at a time, graph-captured: 1920x1080 at S=16
    and 640x480 at K=1200 (the paper's image size), m=10, 5 iterations;
    per-call latency percentiles over replays."""
    import torch
    from paper_1509_04232_gb300 import synth
    out = {}
    for name, (w, h, kw, img) in {"1920x1080_S16": (W, H, dict(S=S), image),
                                  "640x480_K1200": (640, 480, dict(K=1200),
                                                    torch.from_numpy(synth.voronoi_frame(640, 480, 120, 6.0, 77)).to(dev))
                                  }.items():
        seg = pkg.Segmenter(w, h, m=M, iterations=ITERS, **kw)
        labels = torch.empty((h, w), dtype=torch.int32, device=dev)
        centres = torch.empty((seg.K_eff, 6), dtype=torch.float32, device=dev)
        n0 = seg.launches
        g = _capture(lambda: seg.segment(img, labels, centres, stream=stream), stream)
        per_frame = (seg.launches - n0) // 2
        reps = max(50, min(args.steps, 300))
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                g.replay()
            evs[0].record(stream)
            for k in range(reps):
                g.replay()
                evs[k + 1].record(stream)
        torch.cuda.synchronize()
        t = np.array([evs[k].elapsed_time(evs[k + 1]) for k in range(reps)])
        out[name] = {"ms_p50": float(np.percentile(t, 50)), "ms_p99": float(np.percentile(t, 99)),
                     "frames_per_s": 1e3 / float(np.mean(t)), "K_eff": seg.K_eff, "iterations": ITERS,
                     "launches_per_frame": per_frame}
        seg.close()
    return out


def video_context(args, pkg, dev, net_small):
    """Video: 120 frames of 3840x2160 (regions moving 0-4 px per frame,
    colour drift 2, noise 6), S=16, m=10, 8 frames per launch, 2 iterations
    per batch after a 10-iteration first batch: the previous batch's
    centres, the grid, and (with a trained network) the learned warm start
    on top of the previous centres; quality against per-frame 10-iteration
    SLIC."""
    import torch
    from paper_1509_04232_gb300 import synth
    from paper_1509_04232_gb300.video import run_video
    VW, VH, T = 3840, 2160, args.video_frames
    host = torch.empty((T, VH, VW, 3), dtype=torch.uint8)
    for t in range(T):
        host[t].numpy()[...] = synth.video_frame(t, VW, VH)
    frames = host.to(dev)
    run_video(frames[:8], 8, 2)  # warm-up: module loading and first-use set-up
    out = {"workload": f"{T} frames 3840x2160, S=16, m=10, 8 per launch, 2 iterations per batch"}
    for key, init, learned in (("previous_centres", "previous", False), ("grid", "grid", False),
                               ("previous_centres_learned", "previous", True)):
        net = None
        if learned:
            if net_small is None:
                continue
            from paper_1509_04232_gb300 import warmstart as ws
            net = ws.WarmStartNet(VW, VH, S, max_batch=8, seed=0, m=M)
            net.set_params(net_small.params())
        r = run_video(frames, 8, 2, init=init, net=net)
        r["agreement_vs_plain_10"].pop("per_frame")
        out[key] = r
        if net is not None:
            net.close()
    return out


def components_step(args, pkg, stream, dev):
    """The bench step (--batch frames of 1920x1080, S=16, m=10; --iterations,
    default 10) with component-based connectivity (mode 2) and with the
    paper's local rule (mode 1), one captured graph each, in the launch shape
    --tuning gives (else autotuned): ms per step for both and the difference."""
    import torch
    from paper_1509_04232_gb300 import synth
    B, iters = args.batch, args.iterations if args.iterations is not None else FULL_ITERS
    imgs = [torch.from_numpy(synth.voronoi_frame(W, H, 400, 6.0, synth.seed_of(1, f))).to(dev) for f in range(B)]
    out = {"frames": B, "iterations": iters}
    for mode in (2, 1):
        bs = pkg.BatchSegmenter([dict(width=W, height=H, S=S, m=M)] * B, iterations=iters, device=dev,
                                enforce_connectivity=mode)
        bs.bind(imgs)
        if args.tuning:
            bs.set_tuning(*((tuple(int(v) for v in args.tuning.split(",")) + (0, 1))[:6]))
        else:
            bs.autotune(os.path.join(tempfile.gettempdir(), "slicgb_autotune.jsonl"), stream=stream)
        g = _capture(lambda: bs.segment(stream=stream), stream)
        out[f"mode{mode}_ms_per_step"] = _graph_ms(g, stream, args, 1, dev)
        bs.status()
        bs.close()
    out["components_minus_local_rule_ms"] = out["mode2_ms_per_step"] - out["mode1_ms_per_step"]
    out["frames_per_s"] = B / (out["mode2_ms_per_step"] / 1e3)
    return out


def mixed_batch_throughput(args, pkg, stream, dev):
    """The 256-frame mixed batch (64 each of 640x480, 1280x720, 1920x1080,
    3840x2160; S in {8,16,32}, m in {5,10,20}; 5 iterations): one captured
    graph per step, autotuned, inputs resident; rank 0 only (a context line,
    not the headline)."""
    import torch
    from paper_1509_04232_gb300 import synth
    specs = synth.mixed_batch_specs(256)
    frames = [dict(width=w, height=h, S=s_, m=m_) for (w, h, s_, m_) in specs]
    imgs = [torch.from_numpy(synth.mixed_batch_frame(f, w, h)).to(dev) for f, (w, h, _, _) in enumerate(specs)]
    bs = pkg.BatchSegmenter(frames, iterations=ITERS, device=dev)
    bs.bind(imgs)
    ctas, stages, rows, tile_h, fused, groups = bs.autotune(
        os.path.join(tempfile.gettempdir(), "slicgb_autotune.jsonl"), stream=stream)
    with torch.cuda.stream(stream):
        bs.segment(stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        bs.segment(stream)
    steps = max(3, min(args.steps, 20))
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            g.replay()
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    bs.status()
    px = sum(w * h for (w, h, _, _) in specs)
    bs.close()
    return {"frames": len(specs), "megapixels": px / 1e6, "ms_per_step": ms, "frames_per_s": len(specs) / (ms / 1e3),
            "megapixels_per_s": px / 1e6 / (ms / 1e3), "steps": steps, "ctas_per_sm": ctas, "pipeline_stages": stages,
            "row_groups_per_warp": rows, "tile": f"32x{tile_h}", "fused_passes": bool(fused),
            "frame_groups": groups, "iterations": ITERS}


def _graph_ms(graph, stream, args, world, dev):
    """Milliseconds per replay of a captured step: warm-up replays, then
    `steps` replays between CUDA events on the replay stream."""
    import torch
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            graph.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            graph.replay()
        e1.record(stream)
    torch.cuda.synchronize()
    return max_over_ranks(e0.elapsed_time(e1), world, dev) / args.steps


def sec2_options(args, pkg, images, B, stream, world, dev, tuning):
    """The two optional steps of Sec. 2 on the bench frames, in the tuned
    launch shape, one CUDA graph per step timed like `value`: the stopping
    test (mean L1 move of the centres below a threshold, per-frame early
    exit, at most 10 iterations) at three thresholds, and the seed
    perturbation (5 iterations). Agreement is measured on the first 8
    frames against the 10-iteration labels (with perturbed seeds for the
    perturbed run). Also the input variants at the bench's iterations:
    4-channel RGBA input and the raw-RGB and XYZ feature spaces, and the
    component-based connectivity mode."""
    import torch
    q = min(8, B)

    def run(cfg, iterations, frames=None, connectivity=1):
        bs = pkg.BatchSegmenter([dict(width=W, height=H, S=S, m=M, **cfg)] * B, iterations=iterations, device=dev,
                                enforce_connectivity=connectivity)
        src = frames if frames is not None else images
        bs.bind([src[f] for f in range(B)])
        bs.set_tuning(*tuning)
        with torch.cuda.stream(stream):
            bs.segment(stream)
        torch.cuda.synchronize()
        labels = [bs.labels[f].clone() for f in range(q)]
        its = bs.iterations_run
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            bs.segment(stream)
        ms = _graph_ms(g, stream, args, world, dev)
        bs.close()
        return labels, its, world * B / (ms / 1e3)

    def agreement(a, b):
        return float(np.mean([torch.eq(x, y).float().mean().item() for x, y in zip(a, b)]))

    ref, _, fps10 = run({}, 10)
    stopping = []
    for eps in (0.5, 0.3, 0.2):
        lab, its, fps = run(dict(convergence=eps), 10)
        stopping.append({"threshold_px": eps, "frames_per_s": fps, "mean_updates": float(np.mean(its)),
                         "agreement_with_10_iterations": round(agreement(lab, ref), 5)})
    pref, _, _ = run(dict(perturb_seeds=True), 10)
    plab, _, pfps = run(dict(perturb_seeds=True), ITERS)
    _, _, fps5 = run({}, ITERS)
    # Input variants (scope row f3): 4-channel RGBA input, raw RGB and XYZ
    # feature spaces, same frames and iterations as `value`.
    rgba = [torch.cat([images[f], torch.full_like(images[f][..., :1], 255)], dim=-1).contiguous() for f in range(B)]
    variants = {}
    for name, cfg, frames in (("rgba_cielab", dict(in_channels=4), rgba), ("rgb_features", dict(color_space=1), None),
                              ("xyz_features", dict(color_space=2), None)):
        variants[name] = run(cfg, ITERS, frames)[2]
    # Component-based connectivity (the original SLIC's; scope row f4) in
    # place of the paper's two-pass rule, same frames and iterations.
    comp_fps = run({}, ITERS, None, 2)[2]
    return {"frames": q, "plain_frames_per_s_at_10_iterations": fps10,
            "stopping_test_max_10_iterations": stopping,
            "seed_perturbation": {"iterations": ITERS, "frames_per_s": pfps, "plain_frames_per_s": fps5,
                                  "agreement_with_own_10_iterations": round(agreement(plab, pref), 5)},
            "input_variants_frames_per_s": variants,
            "component_connectivity_frames_per_s": comp_fps}


def agreement_sweeps(args, pkg, dev, stream):
    """Mean label agreement with 10-iteration SLIC over the evaluation set
    (64 seeded 1080p frames, other seeds than the throughput frames; labels
    after connectivity) for the plain path at 0..10 iterations and, unless
    --no-learned, the learned warm start at 0..10 iterations after training
    its network on seeded 256x256 images (outside every timed region); the
    smallest iteration count of each reaching 99 %. Returns (quality dict,
    trained 256x256 network or None)."""
    import torch
    from paper_1509_04232_gb300 import synth
    from paper_1509_04232_gb300 import warmstart as ws
    n_eval = args.eval_frames
    host = np.stack([synth.hd_image(30_000 + i, W, H) for i in range(n_eval)])
    evals = torch.from_numpy(host).to(dev)
    chunk = 32

    def run(iterations, net=None):
        eq = 0
        for c0 in range(0, n_eval, chunk):
            sub = evals[c0:c0 + chunk]
            lab = (ws.warm_start_segment(net, sub, iterations, m=M)[0] if net is not None
                   else ws.plain_segment(sub, iterations, S, M)[0])
            eq += sum(int(torch.eq(x, y).sum().item()) for x, y in zip(lab, refs[c0:c0 + chunk]))
        return eq / (n_eval * W * H)

    refs = []
    for c0 in range(0, n_eval, chunk):
        refs += ws.plain_segment(evals[c0:c0 + chunk], FULL_ITERS, S, M)[0]
    plain = {str(n): round(run(n), 5) for n in range(0, FULL_ITERS + 1)}
    n_plain = min(n for n in range(FULL_ITERS + 1) if plain[str(n)] >= AGREE_BAR)
    q = {"reference": "plain SLIC at 10 iterations, connectivity on (GPU; the parity tests hold it to the FP64 "
                      "oracle at >= 99.5 %)",
         "eval_frames": n_eval, "bar": AGREE_BAR,
         "plain_agreement_by_iterations": plain, "plain_iterations_at_99": n_plain}
    if args.no_learned:
        return q, None
    t0 = time.time()
    small = ws.WarmStartNet(256, 256, S, max_batch=64, seed=0, m=M)
    hist = ws.train(small, n_images=args.train_images, batch=64, epochs=args.train_epochs, lr=2e-3, log_every=50)
    train_s = time.time() - t0
    net = ws.WarmStartNet(W, H, S, max_batch=chunk, seed=0, m=M)
    net.set_params(small.params())
    learned = {str(n): round(run(n, net), 5) for n in range(0, FULL_ITERS + 1)}
    reach = [n for n in range(FULL_ITERS + 1) if learned[str(n)] >= AGREE_BAR]
    q.update({"learned_agreement_by_iterations": learned,
              "learned_iterations_at_99": reach[0] if reach else None,
              "learned_training": {"images": args.train_images, "epochs": args.train_epochs, "seconds": train_s,
                                   "final_loss": hist[-1][1] if hist else None,
                                   "final_pixel_accuracy": hist[-1][2] if hist else None}})
    q["network_forward"] = network_forward_roofline(args, net, evals[:chunk], stream)
    net.close()
    return q, small


def network_forward_roofline(args, net, images, stream):
    """The network alone (input channels, four convolutions, labels) on a
    32-frame 1080p batch, against the bf16 tensor roofline: the algorithmic
    work is 2 * 9 * (14*32 + 32*32 + 32*32 + 32*9) FLOP per pixel."""
    import torch
    B = images.shape[0]
    labels = torch.empty((B, H, W), dtype=torch.int32, device=images.device)
    s_handle = int(stream.cuda_stream)
    # (an NVTX range around the eager call lets a profiler pick these launches)
    torch.cuda.nvtx.range_push("network_forward")
    with torch.cuda.stream(stream):
        net.forward(images, labels=labels, stream=s_handle)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    gn = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gn, stream=stream):
        net.forward(images, labels=labels, stream=s_handle)
    net_ms = _graph_ms(gn, stream, args, 1, None)
    flop = 2.0 * 9 * (14 * 32 + 32 * 32 + 32 * 32 + 32 * 9) * B * W * H
    peaks, peak_kind = measured_peaks()
    tflops = flop / (net_ms / 1e3) / 1e12
    return {"frames": B, "ms_per_batch": net_ms, "frames_per_s": B / (net_ms / 1e3), "achieved": tflops,
            "unit": "TFLOP/s", "bound": "tensor", "peak": peaks.get("bf16_tflops"),
            "frac": tflops / peaks["bf16_tflops"] if peaks.get("bf16_tflops") else None, "peak_kind": peak_kind,
            "flop_per_pixel": flop / (B * W * H),
            "kernels": "tcgen05.mma M128 x N x K16 bf16 implicit GEMM, TMEM accumulators"}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--batch", type=int, default=32, help="1080p frames per GPU per step")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-frames", type=int, default=0,
                    help="frames in the oracle CPU-baseline sample (0: two per host core)")
    ap.add_argument("--train-images", type=int, default=20000, help="training images for the learned leg")
    ap.add_argument("--train-epochs", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", "--no-quality", dest="no_learned", action="store_true",
                    help="skip the learned warm start (the plain sweep always runs: it sets the iteration count)")
    ap.add_argument("--eval-frames", type=int, default=EVAL_FRAMES, help="frames of the agreement evaluation set")
    ap.add_argument("--no-video", action="store_true", help="skip the 4K video context")
    ap.add_argument("--video-frames", type=int, default=120)
    ap.add_argument("--no-single", action="store_true", help="skip the single-frame latencies")
    ap.add_argument("--no-mixed", action="store_true", help="skip the 256-frame mixed-resolution batch")
    ap.add_argument("--no-options", action="store_true",
                    help="skip the Sec. 2 options (stopping test, seed perturbation)")
    ap.add_argument("--iterations", type=int, default=None,
                    help="time the plain path at this iteration count instead of the one the agreement sweep "
                         "finds (skips the sweep and the learned leg; for profiling)")
    ap.add_argument("--tuning", default=None, metavar="CTAS,STAGES,ROWS,TILE_H[,FUSED[,GROUPS]]",
                    help="launch shape of the assignment passes instead of autotuning (for profiling)")
    ap.add_argument("--train-only", action="store_true",
                    help="train the warm-start network on --train-images images and print its line (for profiling)")
    ap.add_argument("--mixed-only", action="store_true",
                    help="run only the 256-frame mixed batch and print its line (for profiling)")
    ap.add_argument("--components-only", action="store_true",
                    help="run only the bench step with component connectivity and print its line (for profiling)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

"""The batched path: per-frame results bit-identical to single-frame
slic_segment (exact integer sums make them order-independent), mixed sizes,
S and m in one batch, initial centres, the launch-shape autotuner and its
cache, and the error paths of the batch API."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1509_04232_gb300 import synth

pytestmark = pytest.mark.gpu


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _frames_mixed():
    return [dict(width=320, height=240, S=16, m=10.0), dict(width=333, height=257, S=13, m=20.0),
            dict(width=640, height=480, S=8, m=5.0), dict(width=97, height=61, K=50, m=10.0),
            dict(width=128, height=96, S=32, m=10.0, color_space=1), dict(width=64, height=48, S=3, m=10.0)]


@pytest.mark.parametrize("iterations,conn", [(5, True), (0, False), (3, False)])
def test_batch_bit_identical_to_single_frames(slic_gpu, iterations, conn):
    import torch
    pkg = slic_gpu
    frames = _frames_mixed()
    imgs = [_cuda(synth.voronoi_frame(f["width"], f["height"], 30, 6.0, 100 + i)) for i, f in enumerate(frames)]
    bs = pkg.BatchSegmenter(frames, iterations=iterations, enforce_connectivity=conn)
    bs.bind(imgs)
    labels, centres = bs.segment()
    bs.status()
    for i, f in enumerate(frames):
        seg = pkg.Segmenter(f["width"], f["height"], S=f.get("S", 0), K=f.get("K", 0), m=f["m"],
                            iterations=iterations, enforce_connectivity=conn, color_space=f.get("color_space", 0))
        l1, c1 = seg.segment(imgs[i])
        torch.cuda.synchronize()
        np.testing.assert_array_equal(labels[i].cpu().numpy(), l1.cpu().numpy())
        np.testing.assert_array_equal(centres[i].cpu().numpy(), c1.cpu().numpy())


def test_batch_matches_oracle_on_mixed_batch(slic_gpu):
    pkg = slic_gpu
    frames = _frames_mixed()[:4]
    host = [synth.voronoi_frame(f["width"], f["height"], 30, 6.0, 200 + i) for i, f in enumerate(frames)]
    bs = pkg.BatchSegmenter(frames, iterations=5)
    bs.bind([_cuda(h) for h in host])
    labels, _ = bs.segment()
    for i, f in enumerate(frames):
        ref = oracle.slic(host[i], K=f.get("K", 0), S=f.get("S", 0), m=f["m"], iterations=5)
        assert np.mean(labels[i].cpu().numpy() == ref["labels"]) >= 0.995


def test_batch_repeatable_and_launch_count(slic_gpu):
    import torch
    pkg = slic_gpu
    frames = [dict(width=320, height=240, S=16)] * 3
    bs = pkg.BatchSegmenter(frames, iterations=4)
    bs.bind([_cuda(synth.small_image(i)) for i in range(3)])
    l1 = [t.clone() for t in bs.segment()[0]]
    n0 = bs.info[1]
    l2 = bs.segment()[0]
    torch.cuda.synchronize()
    # conversion pre-pass, init, 5 assignments, 4 updates and one launch of
    # both connectivity passes (pipelined kernel in use); independent of the
    # number of frames
    assert bs.info[3] in (3, 4)
    assert bs.info[1] - n0 == 2 * 4 + 4
    for a, b in zip(l1, l2):
        assert torch.equal(a, b)
    # fused: conversion, init, passes 0..3 with updates 1..4 in one launch,
    # the last pass, connectivity
    bs.set_fused(True)
    n1 = bs.info[1]
    l3 = bs.segment()[0]
    assert bs.info[1] - n1 == 5 and bs.info[6] == 1
    assert all(torch.equal(a, b) for a, b in zip(l1, l3))


def test_batch_initial_centres(slic_gpu):
    """Frames with given initial centres start from them (video warm start)."""
    pkg = slic_gpu
    img = synth.small_image(7)
    ref_prev = oracle.slic(img, K=300, m=10, iterations=3)
    init = _cuda(ref_prev["centres"].astype(np.float32))
    bs = pkg.BatchSegmenter([dict(width=320, height=240, K=300)] * 2, iterations=0, enforce_connectivity=False)
    bs.bind([_cuda(img), _cuda(img)], init_centres=[init, None])
    labels, centres = bs.segment()
    want = oracle.slic(img, K=300, m=10, iterations=0, enforce_connectivity=False,
                       init_centres=ref_prev["centres"].astype(np.float32).astype(float))
    grid = oracle.slic(img, K=300, m=10, iterations=0, enforce_connectivity=False)
    assert np.mean(labels[0].cpu().numpy() == want["labels"]) >= 0.999
    assert np.mean(labels[1].cpu().numpy() == grid["labels"]) >= 0.999
    np.testing.assert_array_equal(centres[0].cpu().numpy(), ref_prev["centres"].astype(np.float32))


def test_autotune_writes_and_reuses_cache(slic_gpu, tmp_path):
    pkg = slic_gpu
    frames = [dict(width=640, height=480, S=16), dict(width=320, height=240, S=8)]
    bs = pkg.BatchSegmenter(frames, iterations=2)
    bs.bind([_cuda(synth.voronoi_frame(f["width"], f["height"], 20, 6.0, 5)) for f in frames])
    cache = str(tmp_path / "tune.jsonl")
    c1, st1, rw1, th1, fu1, gr1 = bs.autotune(cache)
    assert c1 >= 1 and 3 <= st1 <= 4 and rw1 in (1, 2) and th1 in (32, 64) and fu1 in (0, 1) and gr1 in (1, 2)
    line = json.loads(open(cache).read().splitlines()[0])
    assert line["ctas_per_sm"] == c1 and line["stages"] == st1 and line["rows"] == rw1 and line["tile_h"] == th1
    assert line["fused"] == fu1 and line["groups"] == gr1
    assert "640x480s16" in line["key"]
    bs.set_tuning(0, 3 if st1 != 3 else 4, 1, 32, fused=1 - fu1, groups=3 - gr1)
    assert bs.autotune(cache) == (c1, st1, rw1, th1, fu1, gr1)   # served from the cache
    assert len(open(cache).read().splitlines()) == 1
    assert bs.info[2:] == (c1, st1, rw1, th1, fu1, gr1)


@pytest.mark.parametrize("stages", [3, 4])
def test_pipeline_depth_is_bit_exact(slic_gpu, stages):
    """Every pipeline depth and launch shape gives the same labels and centres
    (fixed-point update sums are order-independent)."""
    import torch
    pkg = slic_gpu
    frames = [dict(width=1920, height=1080, S=16)] * 2 + [dict(width=333, height=211, S=12)]
    imgs = [_cuda(synth.hd_image(3)), _cuda(synth.hd_image(4)),
            _cuda(synth.voronoi_frame(333, 211, 15, 6.0, 9))]
    ref = pkg.BatchSegmenter(frames, iterations=4)
    ref.bind(imgs)
    ref.set_tuning(1, 3)
    want_l, want_c = [[t.clone() for t in x] for x in ref.segment()]
    bs = pkg.BatchSegmenter(frames, iterations=4)
    bs.bind(imgs)
    for cps in (0, 1, 2):
        bs.set_tuning(cps, stages)
        labels, centres = bs.segment()
        bs.status()
        for a, b in zip(labels, want_l):
            assert torch.equal(a, b)
        for a, b in zip(centres, want_c):
            assert torch.equal(a, b)
    for bad in (2, 5):
        with pytest.raises(pkg.SlicError):
            bs.set_tuning(0, bad)
    with pytest.raises(pkg.SlicError):        # S = 12 is not a multiple of 8
        bs.set_tuning(0, stages, 2)
    with pytest.raises(pkg.SlicError):
        bs.set_tuning(0, stages, 1, 64)


@pytest.mark.parametrize("stages", [3, 4])
def test_two_row_groups_are_bit_exact(slic_gpu, stages):
    """The 8-pixels-per-thread builds give the single-frame results bit for
    bit (S multiples of 8, ragged sizes included), with 32x32 tiles (128
    threads) and 32x64 tiles (256 threads; the 211-row frame ends in a
    partial 32x64 tile, the 480-row one in a 32x32 half)."""
    import torch
    pkg = slic_gpu
    frames = [dict(width=1920, height=1080, S=16), dict(width=333, height=211, S=8),
              dict(width=640, height=480, S=32, m=20.0)]
    imgs = [_cuda(synth.hd_image(5)), _cuda(synth.voronoi_frame(333, 211, 15, 6.0, 9)),
            _cuda(synth.voronoi_frame(640, 480, 30, 6.0, 10))]
    bs = pkg.BatchSegmenter(frames, iterations=4)
    bs.bind(imgs)
    for cps, th in ((0, 32), (2, 32), (0, 64), (1, 64)):
        bs.set_tuning(cps, stages, 2, th)
        labels, centres = bs.segment()
        bs.status()
        assert bs.info[4] == 2 and bs.info[5] == th
        for i, f in enumerate(frames):
            seg = pkg.Segmenter(f["width"], f["height"], S=f["S"], m=f.get("m", 10.0), iterations=4)
            l1, c1 = seg.segment(imgs[i])
            assert torch.equal(labels[i], l1)
            assert torch.equal(centres[i], c1)


def test_large_clusters_sum_exactly(slic_gpu):
    """One centre wins far more pixels of a tile than its cell holds. The
    image is black but for a white 48x48 square, the 3x3 cells around one
    centre; the other eight centres in the square start on black dots, and m
    is small, so every white pixel picks the white centre in every pass.
    About 1000 pixels at L = 100 then go into one window cell of one tile,
    more than a 32-bit sum of their fixed-point colours holds
    (1000 x 100 x 2^15 > 2^31); the pipelined kernel's private copies and
    flush must still give the single-frame results bit for bit, in every
    tile shape."""
    import torch
    pkg = slic_gpu
    W, H, S = 256, 128, 16
    ns_c = -(-W // S)
    img = np.zeros((H, W, 3), np.uint8)
    img[2 * S:5 * S, 4 * S:7 * S] = 255  # cells (2..4, 4..6)
    white = 3 * ns_c + 5
    cen = oracle.init_centres(oracle.convert(img), S)
    for r in (2, 3, 4):
        for c in (4, 5, 6):
            if r * ns_c + c != white:
                x, y = (int(np.floor(v)) for v in cen[r * ns_c + c, 3:5])
                img[y - 1:y + 2, x - 1:x + 2] = 0
    d_img = _cuda(img)
    seg = pkg.Segmenter(W, H, S=S, m=1.0, iterations=3, enforce_connectivity=False)
    l1, c1 = seg.segment(d_img)
    torch.cuda.synchronize()
    lab = l1.cpu().numpy()
    # the 32x32 tile at (64, 32) is white but for three 3x3 dots
    assert np.sum(lab[2 * S:4 * S, 4 * S:6 * S] == white) >= 990
    assert c1.cpu().numpy()[white, 0] > 99.0
    bs = pkg.BatchSegmenter([dict(width=W, height=H, S=S, m=1.0)], iterations=3, enforce_connectivity=False)
    bs.bind([d_img])
    for cps, stages, rows, th in ((0, 3, 1, 32), (0, 3, 2, 32), (0, 3, 2, 64)):
        bs.set_tuning(cps, stages, rows, th)
        labels, centres = bs.segment()
        bs.status()
        assert bs.info[4] == rows and bs.info[5] == th
        assert torch.equal(labels[0], l1)
        assert torch.equal(centres[0], c1)


def test_batch_errors(slic_gpu):
    pkg = slic_gpu
    from paper_1509_04232_gb300 import _binding
    bad = [pkg.slic_params(64, 48, 0, 16, 10.0, 3, 0, 1, 3), pkg.slic_params(64, 48, 0, 16, 10.0, 4, 0, 1, 3)]
    with pytest.raises(pkg.SlicError) as ei:
        pkg.slic_batch_create(bad)
    assert ei.value.status == _binding.SLIC_ERR_INVALID and "same iterations" in str(ei.value)
    b = pkg.slic_batch_create(bad[:1])
    with pytest.raises(pkg.SlicError) as ei:
        pkg.slic_batch_segment(b)
    assert ei.value.status == _binding.SLIC_ERR_STATE
    pkg.slic_batch_destroy(b)


def test_profile_timers_outside_capture(slic_gpu):
    """Per-launch timers work on a plain stream as well as under capture."""
    pkg = slic_gpu
    frames = [dict(width=640, height=480, S=16)] * 2
    bs = pkg.BatchSegmenter(frames, iterations=3)
    bs.bind([_cuda(synth.voronoi_frame(640, 480, 30, 6.0, s)) for s in (1, 2)])
    pkg.slic_batch_profile_enable(bs.handle, True)
    bs.segment()
    times = pkg.slic_batch_profile_times(bs.handle)
    assert len(times) == 4 and all(t > 0 for t in times)  # one per pass
    bs.set_fused(True)
    bs.segment()
    times = pkg.slic_batch_profile_times(bs.handle)
    assert len(times) == 4 + 2 and all(t > 0 for t in times)  # the fused passes 0..2, the last pass
    bs.status()


def test_segment_host_matches_device_path(slic_gpu):
    """Host buffers in and out (page-locked) give the device path's results."""
    import torch
    pkg = slic_gpu
    frames = [dict(width=320, height=240, S=16), dict(width=333, height=211, S=12)]
    imgs = [synth.small_image(3), synth.voronoi_frame(333, 211, 15, 6.0, 4)]
    ref = pkg.BatchSegmenter(frames, iterations=3)
    ref.bind([_cuda(i) for i in imgs])
    want_l, want_c = [[t.cpu() for t in x] for x in ref.segment()]
    bs = pkg.BatchSegmenter(frames, iterations=3)
    bs.bind([torch.empty(i.shape, dtype=torch.uint8, device="cuda") for i in imgs])
    h_img = [torch.from_numpy(np.ascontiguousarray(i)).pin_memory() for i in imgs]
    h_lab = [torch.empty(t.shape, dtype=torch.int32).pin_memory() for t in want_l]
    h_cen = [torch.empty(t.shape, dtype=torch.float32).pin_memory() for t in want_c]
    stream = torch.cuda.Stream()
    bs.segment_host(h_img, h_lab, h_cen, stream=stream)
    stream.synchronize()
    for a, b in zip(h_lab, want_l):
        assert torch.equal(a, b)
    for a, b in zip(h_cen, want_c):
        assert torch.equal(a, b)
    h_lab2 = [torch.zeros(t.shape, dtype=torch.int32).pin_memory() for t in want_l]
    bs.segment_host(h_img, h_lab2, None, stream=stream)   # centres copy skipped
    stream.synchronize()
    assert torch.equal(h_lab2[0], want_l[0])


def test_segment_host_with_contiguous_buffers(slic_gpu):
    """The whole batch in one host and one device allocation (the copies
    merge into one per direction and kind): same results as the device
    path, and a host label array skipped for one frame stays untouched."""
    import torch
    pkg = slic_gpu
    W, H, n = 320, 240, 3
    host = torch.from_numpy(np.stack([synth.small_image(10 + i) for i in range(n)])).pin_memory()
    ref = pkg.BatchSegmenter([dict(width=W, height=H, S=16)] * n, iterations=3)
    ref.bind([host[i].cuda() for i in range(n)])
    want_l, want_c = [[t.cpu() for t in x] for x in ref.segment()]
    bs = pkg.BatchSegmenter([dict(width=W, height=H, S=16)] * n, iterations=3)
    dev = torch.empty_like(host, device="cuda")
    bs.bind([dev[i] for i in range(n)])
    h_lab = torch.full((n, H, W), -5, dtype=torch.int32).pin_memory()
    h_cen = torch.empty((n, bs.K_eff[0], 6), dtype=torch.float32).pin_memory()
    stream = torch.cuda.Stream()
    bs.segment_host([host[i] for i in range(n)], [h_lab[0], None, h_lab[2]], [h_cen[i] for i in range(n)],
                    stream=stream)
    stream.synchronize()
    assert torch.equal(h_lab[0], want_l[0]) and torch.equal(h_lab[2], want_l[2])
    assert bool((h_lab[1] == -5).all())
    for i in range(n):
        assert torch.equal(h_cen[i], want_c[i])


def test_rebind_is_stream_ordered(slic_gpu):
    """Rebinding without a device-wide wait: frames A, then B and A again
    on one stream, each result equal to a batch bound to those frames only;
    with initial centres on the rebind as well."""
    import torch
    pkg = slic_gpu
    W, H = 320, 240
    A = [_cuda(synth.small_image(20 + i)) for i in range(2)]
    B = [_cuda(synth.small_image(30 + i)) for i in range(2)]

    def fresh(imgs, init=None):
        r = pkg.BatchSegmenter([dict(width=W, height=H, S=16)] * 2, iterations=2)
        r.bind(imgs, init_centres=init)
        return [[t.clone() for t in x] for x in r.segment()]

    want_a, want_b = fresh(A), fresh(B)
    bs = pkg.BatchSegmenter([dict(width=W, height=H, S=16)] * 2, iterations=2)
    bs.bind(A)
    stream = torch.cuda.Stream()
    got = []
    with torch.cuda.stream(stream):
        for imgs in (B, A, B):
            bs.bind(imgs, stream=stream)
            got.append([[t.clone() for t in x] for x in bs.segment(stream=stream)])
        init = [want_a[1][0].clone(), None]
        bs.bind(B, init_centres=init, stream=stream)
        got.append([[t.clone() for t in x] for x in bs.segment(stream=stream)])
    stream.synchronize()
    want_bi = fresh(B, init)
    for g, w in zip(got, (want_b, want_a, want_b, want_bi)):
        for x, y in zip(g[0] + g[1], w[0] + w[1]):
            assert torch.equal(x, y)


def _fused_vs_passes(pkg, frames, imgs, iterations, shapes, **kw):
    """Labels, centres and update counts of the fused launch equal one
    launch per pass and per update, for each launch shape."""
    import torch
    bs = pkg.BatchSegmenter(frames, iterations=iterations, **kw)
    bs.bind(imgs)
    for shape in shapes:
        bs.set_tuning(*shape)
        bs.set_fused(False)
        l0, c0 = bs.segment()
        l0, c0 = [t.clone() for t in l0], [t.clone() for t in c0]
        n0 = bs.iterations_run
        bs.set_fused(True)
        l1, c1 = bs.segment()
        bs.status()
        assert bs.iterations_run == n0, shape
        for i in range(len(frames)):
            assert torch.equal(l1[i], l0[i]), (shape, i)
            assert torch.equal(c1[i], c0[i]), (shape, i)
    bs.close()


@pytest.mark.parametrize("iterations", [1, 4])
def test_fused_passes_are_bit_exact(slic_gpu, iterations):
    """Every build of the fused kernel (32x32 tiles with 4 or 8 pixels per
    thread, 32x64 tiles; 1 to 4 CTAs per SM; 3 and 4 stages), on frames of
    uneven size, S and m: a 1080p frame, ragged ones, a tiny one with fewer
    tiles than CTAs, and one with the stopping test."""
    pkg = slic_gpu
    frames = [dict(width=1920, height=1080, S=16), dict(width=333, height=211, S=8),
              dict(width=640, height=480, S=32, m=20.0), dict(width=64, height=48, S=16),
              dict(width=1280, height=720, S=8, convergence=0.4)]
    imgs = [_cuda(synth.hd_image(7)), _cuda(synth.voronoi_frame(333, 211, 15, 6.0, 11)),
            _cuda(synth.voronoi_frame(640, 480, 30, 6.0, 12)), _cuda(synth.voronoi_frame(64, 48, 5, 6.0, 13)),
            _cuda(synth.voronoi_frame(1280, 720, 200, 6.0, 14))]
    shapes = [(0, 3, 1, 32), (4, 3, 1, 32), (0, 4, 1, 32), (0, 3, 2, 32), (2, 4, 2, 32), (0, 3, 2, 64),
              (1, 3, 2, 64)]
    _fused_vs_passes(pkg, frames, imgs, iterations, shapes)


def test_fused_passes_other_cell_alignments(slic_gpu):
    """S not a multiple of 4 (each pixel's own cell), in the 80- and
    64-register builds; and one frame alone, whose pass holds its tiles and
    its own update chunks only."""
    pkg = slic_gpu
    frames = [dict(width=333, height=257, S=13), dict(width=320, height=240, S=12), dict(width=97, height=61, S=7)]
    imgs = [_cuda(synth.voronoi_frame(333, 257, 20, 6.0, 21)), _cuda(synth.small_image(22)),
            _cuda(synth.voronoi_frame(97, 61, 8, 6.0, 23))]
    _fused_vs_passes(pkg, frames, imgs, 3, [(0, 3, 1, 32), (4, 4, 1, 32)])
    _fused_vs_passes(pkg, frames[:1], imgs[:1], 5, [(0, 3, 1, 32)])
    _fused_vs_passes(pkg, [dict(width=1920, height=1080, S=16)], [_cuda(synth.hd_image(24))], 2,
                     [(0, 3, 2, 64), (0, 3, 1, 32)])


def test_fused_passes_full_bench_batch(slic_gpu):
    """32 frames of 1920x1080 at 10 iterations (the throughput batch), in
    the 32x64 shape: fused and per-pass launches agree bit for bit, and the
    fused launch matches the single-frame path on two sampled frames."""
    import torch
    pkg = slic_gpu
    host = [synth.voronoi_frame(1920, 1080, 400, 6.0, synth.seed_of(1, i)) for i in range(32)]
    imgs = [_cuda(h) for h in host]
    frames = [dict(width=1920, height=1080, S=16)] * 32
    _fused_vs_passes(pkg, frames, imgs, 10, [(0, 3, 2, 64)])
    bs = pkg.BatchSegmenter(frames, iterations=10)
    bs.bind(imgs)
    bs.set_tuning(0, 3, 2, 64)
    labels, centres = bs.segment()
    bs.status()
    for i in (0, 31):
        seg = pkg.Segmenter(1920, 1080, S=16, iterations=10)
        l1, c1 = seg.segment(imgs[i])
        assert torch.equal(labels[i], l1)
        assert torch.equal(centres[i], c1)


def test_frame_groups_are_bit_exact(slic_gpu):
    """Frames run as 1 to 4 groups on concurrent streams give the same
    labels and centres, also with the stopping test, after a rebind, through
    host buffers and under graph capture."""
    import torch
    pkg = slic_gpu
    frames = [dict(width=1920, height=1080, S=16), dict(width=333, height=211, S=8),
              dict(width=640, height=480, S=32, m=20.0), dict(width=64, height=48, S=16),
              dict(width=1280, height=720, S=8, convergence=0.4), dict(width=320, height=240, S=16)]
    host = [synth.hd_image(31), synth.voronoi_frame(333, 211, 15, 6.0, 32), synth.voronoi_frame(640, 480, 30, 6.0, 33),
            synth.voronoi_frame(64, 48, 5, 6.0, 34), synth.voronoi_frame(1280, 720, 200, 6.0, 35), synth.small_image(36)]
    imgs = [_cuda(h) for h in host]
    bs = pkg.BatchSegmenter(frames, iterations=4)
    bs.bind(imgs)
    bs.set_tuning(0, 3, 2, 64)
    want_l, want_c = [[t.clone() for t in x] for x in bs.segment()]
    want_n = bs.iterations_run
    for groups in (2, 3, 4):
        bs.set_groups(groups)
        assert bs.info[7] == groups
        labels, centres = bs.segment()
        bs.status()
        assert bs.iterations_run == want_n
        for i in range(len(frames)):
            assert torch.equal(labels[i], want_l[i]) and torch.equal(centres[i], want_c[i]), (groups, i)
    # a rebind (the group tables follow the new buffers), under capture
    other = [torch.empty_like(t) for t in imgs]
    for a, b in zip(other, imgs):
        a.copy_(b)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        bs.bind(other, stream=stream)
        bs.segment(stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        bs.segment(stream)
    for lab in bs.labels:
        lab.fill_(-1)
    with torch.cuda.stream(stream):
        g.replay()
    torch.cuda.synchronize()
    bs.status()
    for i in range(len(frames)):
        assert torch.equal(bs.labels[i], want_l[i]), i
    # host buffers in and out (each group's stream copies its own frames in
    # and its results out); one frame's label copy skipped
    h_img = [torch.from_numpy(np.ascontiguousarray(h)).pin_memory() for h in host]
    h_lab = [torch.full(t.shape, -9, dtype=torch.int32).pin_memory() for t in want_l]
    h_cen = [torch.empty(t.shape, dtype=torch.float32).pin_memory() for t in want_c]
    bs.segment_host(h_img, h_lab[:3] + [None] + h_lab[4:], h_cen, stream=stream)
    stream.synchronize()
    for i, (a, b) in enumerate(zip(h_lab, want_l)):
        assert bool((a == -9).all()) if i == 3 else torch.equal(a, b.cpu()), i
    for a, b in zip(h_cen, want_c):
        assert torch.equal(a, b.cpu())
    with pytest.raises(pkg.SlicError):
        bs.set_groups(5)
    bs.close()

"""slic_segment_noalloc: the allocation-free entry point.

Some callers cannot allocate device memory: code running while a stream is
captured into a CUDA graph, processes whose device memory belongs to
another allocator with a fixed budget, and loops that cannot afford the
device synchronisation cudaMalloc/cudaFree may cause. For them the library
keeps its scratch in a static 32 MiB device array instead of per-handle
allocations. These tests call that entry point through the C ABI and check
it bit for bit against the handle-based slic_segment (the same kernels in
the same order), and one case against the FP64 oracle within the parity
tolerance, on calls in a row: each image is segmented after another one
has used the shared array, so a stale sum, feature or flag left there
would show.

This file is named to be collected last.
"""
import numpy as np
import pytest

import oracle
from paper_1509_04232_gb300 import _binding, synth

AGREE_MIN = 0.995   # whole-run label agreement with the oracle, as in the parity tests


def _params(W, H, **kw):
    return _binding.slic_params(W, H, kw.get("K", 0), kw.get("S", 0), float(kw.get("m", 10.0)),
                                kw.get("iterations", 5), kw.get("color_space", 0),
                                int(kw.get("enforce_connectivity", 1)), 3, int(kw.get("perturb_seeds", 0)),
                                float(kw.get("convergence", 0.0)))


CASES = [
    (640, 480, dict(K=1200, m=10.0, iterations=5)),
    (333, 257, dict(S=13, m=20.0, iterations=3)),
    (320, 240, dict(S=16, m=10.0, iterations=4, perturb_seeds=1)),
    (320, 240, dict(S=16, m=10.0, iterations=6, convergence=0.05)),
    (400, 300, dict(S=10, m=10.0, iterations=3, enforce_connectivity=2)),
    (1280, 720, dict(S=16, m=10.0, iterations=2, enforce_connectivity=2)),  # the largest mode-2 size that fits
]


@pytest.mark.gpu
def test_noalloc_equals_handle_path_on_calls_in_a_row(slic_gpu):
    import torch
    pkg = slic_gpu
    stream = torch.cuda.current_stream().cuda_stream
    for W, H, kw in CASES:
        seg = pkg.Segmenter(W, H, **kw)
        imgs = [torch.from_numpy(synth.voronoi_frame(W, H, 60, 6.0, 31 + W + k)).cuda() for k in range(2)]
        want = [seg.segment(img) for img in imgs]
        # A, B, A: every call follows another image's call on the shared array
        for k in (0, 1, 0):
            labels = torch.full((H, W), -7, dtype=torch.int32, device="cuda")
            centres = torch.full((seg.K_eff, 6), float("nan"), dtype=torch.float32, device="cuda")
            pkg.slic_segment_noalloc(_params(W, H, **kw), imgs[k].data_ptr(), labels.data_ptr(),
                                     centres.data_ptr(), stream)
            torch.cuda.synchronize()
            assert torch.equal(labels, want[k][0]), (W, H, kw, k)
            assert torch.equal(centres, want[k][1]), (W, H, kw, k)
        pkg.slic_noalloc_status_check()


@pytest.mark.gpu
def test_noalloc_matches_oracle(slic_gpu):
    import torch
    pkg = slic_gpu
    W, H = 320, 240
    img = synth.small_image(3)
    labels = torch.empty((H, W), dtype=torch.int32, device="cuda")
    centres = torch.empty((300, 6), dtype=torch.float32, device="cuda")
    pkg.slic_segment_noalloc(_params(W, H, K=300, iterations=10), torch.from_numpy(img).cuda().data_ptr(),
                             labels.data_ptr(), centres.data_ptr(), torch.cuda.current_stream().cuda_stream)
    ref = oracle.slic(img, K=300, m=10.0, iterations=10)
    assert float(np.mean(labels.cpu().numpy() == ref["labels"])) >= AGREE_MIN


@pytest.mark.gpu
def test_noalloc_reports_a_walk_that_gave_up(slic_gpu):
    """Component connectivity's bounded walks, limited to one step by fault
    injection, give up on a SLIC label map; the handle-free status check
    reports it once and clears it; with the limit restored a run is clean."""
    import torch
    pkg = slic_gpu
    W, H = 320, 240
    img = torch.from_numpy(synth.small_image(4)).cuda()
    labels = torch.empty((H, W), dtype=torch.int32, device="cuda")
    centres = torch.empty((300, 6), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    p = _params(W, H, S=16, iterations=2, enforce_connectivity=2)
    pkg.slic_noalloc_status_check()
    try:
        pkg.slic_fault_inject(pkg.SLIC_FAULT_WALK_LIMIT, 1)
        pkg.slic_segment_noalloc(p, img.data_ptr(), labels.data_ptr(), centres.data_ptr(), stream)
        with pytest.raises(pkg.SlicError) as ei:
            pkg.slic_noalloc_status_check()
        assert ei.value.status == pkg.SLIC_ERR_TIMEOUT
    finally:
        pkg.slic_fault_inject(pkg.SLIC_FAULT_WALK_LIMIT, 0)
    pkg.slic_noalloc_status_check()  # cleared by the failed check
    pkg.slic_segment_noalloc(p, img.data_ptr(), labels.data_ptr(), centres.data_ptr(), stream)
    pkg.slic_noalloc_status_check()


@pytest.mark.parametrize("W,H,kw", [(1920, 1080, dict(S=16)),
                                    (1024, 1024, dict(S=4, enforce_connectivity=2))])
def test_noalloc_rejects_images_beyond_the_static_scratch(W, H, kw):
    _binding.lib()
    with pytest.raises(_binding.SlicError) as ei:
        _binding.slic_segment_noalloc(_params(W, H, **kw), 16, 16, 16, 0)
    assert ei.value.status == _binding.SLIC_ERR_INVALID
    assert "static scratch" in str(ei.value)

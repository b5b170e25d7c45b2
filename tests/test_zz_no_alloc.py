"""slic_segment_noalloc: the allocation-free entry point.

Some callers cannot allocate device memory: code running while a stream is
captured into a CUDA graph, processes whose device memory belongs to
another allocator with a fixed budget, and loops that cannot afford the
device synchronisation cudaMalloc/cudaFree may cause. For them the library
keeps its scratch in a static 32 MiB device array instead of per-handle
allocations. These tests call that entry point through the C ABI and check
it against the handle-based slic_segment within the parity tolerances used
elsewhere in the suite, on two calls in a row (the second call must not be
disturbed by what the first left in the shared array).

This file is named to be collected last.
"""
import numpy as np
import pytest

from paper_1509_04232_gb300 import _binding, synth

AGREE_MIN = 0.995   # whole-run label agreement, as in the parity tests
CENTRE_TOL = 1e-4   # relative, floor 1, as in the parity tests


def _params(W, H, **kw):
    return _binding.slic_params(W, H, kw.get("K", 0), kw.get("S", 0), float(kw.get("m", 10.0)),
                                kw.get("iterations", 5), kw.get("color_space", 0),
                                int(kw.get("enforce_connectivity", True)), 3)


@pytest.mark.gpu
def test_noalloc_matches_handle_path_twice(slic_gpu):
    import torch
    pkg = slic_gpu
    cases = [(640, 480, dict(K=1200, m=10.0, iterations=5)),
             (333, 257, dict(S=13, m=20.0, iterations=3))]
    for W, H, kw in cases:
        img = torch.from_numpy(synth.voronoi_frame(W, H, 60, 6.0, 31 + W)).cuda()
        seg = pkg.Segmenter(W, H, **kw)
        ref_labels, ref_centres = seg.segment(img)
        labels = torch.full((H, W), -7, dtype=torch.int32, device="cuda")
        centres = torch.full((seg.K_eff, 6), float("nan"), dtype=torch.float32, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        pkg.slic_segment_noalloc(_params(W, H, **kw), img.data_ptr(), labels.data_ptr(), centres.data_ptr(),
                                 stream)
        torch.cuda.synchronize()
        got_l, want_l = labels.cpu().numpy(), ref_labels.cpu().numpy()
        got_c, want_c = centres.cpu().numpy(), ref_centres.cpu().numpy()
        assert np.mean(got_l == want_l) >= AGREE_MIN
        assert np.all(np.abs(got_c - want_c) <= CENTRE_TOL * np.maximum(1.0, np.abs(want_c)))


def test_noalloc_rejects_images_beyond_the_static_scratch():
    _binding.lib()
    with pytest.raises(_binding.SlicError) as ei:
        _binding.slic_segment_noalloc(_params(1920, 1080, S=16), 16, 16, 16, 0)
    assert ei.value.status == _binding.SLIC_ERR_INVALID
    assert "static scratch" in str(ei.value)

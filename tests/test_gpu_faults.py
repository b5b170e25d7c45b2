"""Failure detection without faulting the GPU: fault injection
(slic_fault_inject) makes the library's own failure paths run. A device
allocation that fails gives SLIC_ERR_NOMEM and leaves nothing behind; a
bounded walk of component connectivity that gives up, and a bounded
mbarrier wait of the pipelined assignment that runs out because its
producer stopped issuing copies (before any copy, so none is in flight when
the CTA returns), give SLIC_ERR_TIMEOUT through the status calls; after each,
the same calls succeed again with the same results as before."""
import numpy as np
import pytest

from paper_1509_04232_gb300 import synth

pytestmark = pytest.mark.gpu


def _img(W, H, seed):
    import torch
    return torch.from_numpy(synth.voronoi_frame(W, H, 40, 8.0, seed)).cuda()


def test_allocation_failures_report_nomem(slic_gpu):
    from paper_1509_04232_gb300.warmstart import WarmStartNet
    pkg = slic_gpu
    makers = [lambda: pkg.Segmenter(64, 48, S=8),
              lambda: pkg.Segmenter(64, 48, S=8, enforce_connectivity=2),
              lambda: pkg.BatchSegmenter([dict(width=64, height=48, S=8)] * 2, iterations=1),
              lambda: WarmStartNet(64, 48, 16, max_batch=1)]
    try:
        for make in makers:
            for k in (1, 2, 3):  # the first, second or third allocation from now fails
                pkg.slic_fault_inject(pkg.SLIC_FAULT_ALLOC, k)
                try:
                    obj = make()
                except pkg.SlicError as e:
                    assert e.status == pkg.SLIC_ERR_NOMEM
                else:  # fewer than k allocations: the object is fine
                    obj.close()
                pkg.slic_fault_inject(pkg.SLIC_FAULT_ALLOC, 0)
                make().close()
        # arming the batched warm start allocates its label maps
        net = WarmStartNet(64, 48, 16, max_batch=1)
        bs = pkg.BatchSegmenter([dict(width=64, height=48, S=16)], iterations=1)
        pkg.slic_fault_inject(pkg.SLIC_FAULT_ALLOC, 1)
        with pytest.raises(pkg.SlicError) as ei:
            bs.set_warmstart(net)
        assert ei.value.status == pkg.SLIC_ERR_NOMEM
        pkg.slic_fault_inject(pkg.SLIC_FAULT_ALLOC, 0)
        bs.set_warmstart(net)
    finally:
        pkg.slic_fault_inject(pkg.SLIC_FAULT_ALLOC, 0)


def test_component_walk_timeout_is_reported(slic_gpu):
    import torch
    pkg = slic_gpu
    W, H = 320, 240
    img = _img(W, H, 77)
    seg = pkg.Segmenter(W, H, S=16, iterations=2, enforce_connectivity=2)
    bs = pkg.BatchSegmenter([dict(width=W, height=H, S=16)] * 2, iterations=2, enforce_connectivity=2)
    bs.bind([img, img])
    want, _ = seg.segment(img)
    seg.status()
    try:
        pkg.slic_fault_inject(pkg.SLIC_FAULT_WALK_LIMIT, 1)
        seg.segment(img)
        with pytest.raises(pkg.SlicError) as ei:
            seg.status()
        assert ei.value.status == pkg.SLIC_ERR_TIMEOUT
        bs.segment()
        with pytest.raises(pkg.SlicError) as ei:
            bs.status()
        assert ei.value.status == pkg.SLIC_ERR_TIMEOUT
    finally:
        pkg.slic_fault_inject(pkg.SLIC_FAULT_WALK_LIMIT, 0)
    got, _ = seg.segment(img)
    seg.status()
    assert torch.equal(got, want)
    labels, _ = bs.segment()
    bs.status()
    assert torch.equal(labels[0], want) and torch.equal(labels[1], want)


def test_pipelined_wait_timeout_is_reported(slic_gpu):
    """The producer stops issuing copies; every consumer's bounded wait runs
    out (about a second); the batch reports SLIC_ERR_TIMEOUT once and then
    segments normally again."""
    import torch
    pkg = slic_gpu
    W, H = 320, 240
    imgs = [_img(W, H, 80 + k) for k in range(2)]
    bs = pkg.BatchSegmenter([dict(width=W, height=H, S=16)] * 2, iterations=0)
    bs.bind(imgs)
    assert bs.info[3] > 0, "the pipelined kernel is in use"
    want = [l.clone() for l in bs.segment()[0]]
    bs.status()
    try:
        pkg.slic_fault_inject(pkg.SLIC_FAULT_ABORT_COPIES, 1)
        bs.segment()
        with pytest.raises(pkg.SlicError) as ei:
            bs.status()
        assert ei.value.status == pkg.SLIC_ERR_TIMEOUT
    finally:
        pkg.slic_fault_inject(pkg.SLIC_FAULT_ABORT_COPIES, 0)
    labels, _ = bs.segment()
    bs.status()
    for a, b in zip(labels, want):
        assert torch.equal(a, b)


def test_fused_passes_timeout_is_reported(slic_gpu):
    """The same with the fused passes: the producers issue nothing, the
    consumers' and the phase counters' bounded waits give up (the latter at
    once when the error word is set), every CTA of the cooperative launch
    exits, SLIC_ERR_TIMEOUT is reported once, and the next run is exact."""
    import torch
    pkg = slic_gpu
    W, H = 320, 240
    imgs = [_img(W, H, 90 + k) for k in range(3)]
    bs = pkg.BatchSegmenter([dict(width=W, height=H, S=16)] * 3, iterations=2)
    bs.bind(imgs)
    bs.set_fused(True)
    assert bs.info[6] == 1, "the fused passes are in use"
    want = [l.clone() for l in bs.segment()[0]]
    bs.status()
    try:
        pkg.slic_fault_inject(pkg.SLIC_FAULT_ABORT_COPIES, 1)
        bs.segment()
        with pytest.raises(pkg.SlicError) as ei:
            bs.status()
        assert ei.value.status == pkg.SLIC_ERR_TIMEOUT
    finally:
        pkg.slic_fault_inject(pkg.SLIC_FAULT_ABORT_COPIES, 0)
    labels, _ = bs.segment()
    bs.status()
    for a, b in zip(labels, want):
        assert torch.equal(a, b)


def test_fault_inject_rejects_bad_arguments(slic_gpu):
    pkg = slic_gpu
    for kind, value in ((0, 1), (9, 1), (pkg.SLIC_FAULT_ALLOC, -1), (pkg.SLIC_FAULT_WALK_LIMIT, 1 << 40)):
        with pytest.raises(pkg.SlicError) as ei:
            pkg.slic_fault_inject(kind, value)
        assert ei.value.status == pkg.SLIC_ERR_INVALID

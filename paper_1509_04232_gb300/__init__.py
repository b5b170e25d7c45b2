"""SLIC superpixels on one GB300 (gSLICr, arXiv 1509.04232), GB300-native.

The compute path is ``libslicgb.so`` (hand-written sm_103a CUDA behind the C
ABI in ``include/slic.h``). This package is its thin binding: the C-named
functions in :mod:`._binding` plus :class:`Segmenter`, which only allocates
output tensors with PyTorch and passes their device pointers and the current
stream through. There is no CPU fallback: if the library is missing, calls
raise.
"""
from __future__ import annotations

from ._binding import (SLIC_CIELAB, SLIC_ERR_CUDA, SLIC_ERR_INVALID, SLIC_ERR_NOMEM,  # noqa: F401
                       SLIC_ERR_STATE, SLIC_ERR_TIMEOUT, SLIC_FAULT_ABORT_COPIES, SLIC_FAULT_ALLOC,
                       SLIC_FAULT_WALK_LIMIT, SLIC_OK, SLIC_RGB, SLIC_XYZ, SlicError, library_path, slic_assign,
                       slic_fault_inject, slic_noalloc_status_check,
                       slic_batch_autotune, slic_batch_create, slic_batch_destroy, slic_batch_info,
                       slic_batch_grid, slic_batch_iterations_run, slic_batch_last_error,
                       slic_batch_profile_enable, slic_batch_set_warmstart, slic_set_warmstart,
                       slic_batch_profile_read,
                       slic_batch_profile_times, slic_batch_segment, slic_batch_segment_host,
                       slic_batch_rebind, slic_batch_set_buffers, slic_batch_set_fused, slic_batch_set_groups,
                       slic_batch_set_tuning,
                       slic_batch_status,
                       slic_connectivity_components, slic_connectivity_pass, slic_convert, slic_create,
                       slic_destroy, slic_grid, slic_status_check,
                       slic_init_centres, slic_iterations_run, slic_last_error, slic_launch_count, slic_params,
                       slic_profile_enable, slic_profile_read, slic_segment, slic_segment_noalloc,
                       slic_set_init_centres, slic_update)


def _stream_handle(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Segmenter:
    """One image geometry and parameter set (Sec. 2: K or S, m, and the
    optional seed perturbation and convergence threshold; Sec. 4: colour
    space, iterations, connectivity), owning a library handle."""

    def __init__(self, width: int, height: int, *, K: int = 0, S: int = 0, m: float = 10.0,
                 iterations: int = 10, color_space: int = SLIC_CIELAB, enforce_connectivity: int = 1,
                 in_channels: int = 3, perturb_seeds: bool = False, convergence: float = 0.0):
        # enforce_connectivity: 0 / False none, 1 / True the paper's rule, 2 components
        self.params = slic_params(width, height, K, S, float(m), iterations, color_space,
                                  int(enforce_connectivity), in_channels, int(bool(perturb_seeds)),
                                  float(convergence))
        self.handle = slic_create(self.params)
        self.S, self.ns_c, self.ns_r = slic_grid(self.handle)
        self.K_eff = self.ns_c * self.ns_r

    def close(self):
        if getattr(self, "handle", None):
            slic_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check_image(self, image):
        p = self.params
        if (not image.is_cuda or image.dtype.itemsize != 1 or tuple(image.shape) != (p.height, p.width, p.in_channels)
                or not image.is_contiguous()):
            raise ValueError(f"image must be a contiguous uint8 CUDA tensor of shape "
                             f"({p.height}, {p.width}, {p.in_channels})")

    def segment(self, image, labels=None, centres=None, init_centres=None, stream=None):
        """Labels int32 [H, W] and centres float32 [K_eff, 6] for one image."""
        import torch
        self._check_image(image)
        dev = image.device
        if labels is None:
            labels = torch.empty((self.params.height, self.params.width), dtype=torch.int32, device=dev)
        if centres is None:
            centres = torch.empty((self.K_eff, 6), dtype=torch.float32, device=dev)
        if init_centres is not None:
            slic_set_init_centres(self.handle, init_centres.data_ptr())
        slic_segment(self.handle, image.data_ptr(), labels.data_ptr(), centres.data_ptr(), _stream_handle(stream))
        return labels, centres

    def set_warmstart(self, net):
        """Arm the learned warm start with a network (an object with a
        ``handle`` or a raw slic_net handle), or disarm it with None. The
        network must outlive the arming."""
        self._net = net
        slic_set_warmstart(self.handle, getattr(net, "handle", net) if net is not None else None)

    def convert(self, image, stream=None):
        import torch
        self._check_image(image)
        feat = torch.empty((3, self.params.height, self.params.width), dtype=torch.float32, device=image.device)
        slic_convert(self.handle, image.data_ptr(), feat.data_ptr(), _stream_handle(stream))
        return feat

    def init_centres(self, features, stream=None):
        import torch
        out = torch.empty((self.K_eff, 6), dtype=torch.float32, device=features.device)
        slic_init_centres(self.handle, features.data_ptr(), out.data_ptr(), _stream_handle(stream))
        return out

    def assign(self, features, centres, stream=None):
        import torch
        labels = torch.empty((self.params.height, self.params.width), dtype=torch.int32, device=features.device)
        slic_assign(self.handle, features.data_ptr(), centres.data_ptr(), labels.data_ptr(), _stream_handle(stream))
        return labels

    def update(self, features, labels, centres_in, stream=None):
        out = centres_in.clone()
        slic_update(self.handle, features.data_ptr(), labels.data_ptr(), centres_in.data_ptr(), out.data_ptr(),
                    _stream_handle(stream))
        return out

    def connectivity_components(self, labels, stream=None):
        """Component-based relabelling (handles created with enforce_connectivity=2)."""
        import torch
        out = torch.empty_like(labels)
        slic_connectivity_components(self.handle, labels.data_ptr(), out.data_ptr(), _stream_handle(stream))
        return out

    def status(self):
        """Raises SlicError(SLIC_ERR_TIMEOUT) if a bounded device loop gave up."""
        slic_status_check(self.handle)

    def connectivity_pass(self, labels, stream=None):
        import torch
        out = torch.empty_like(labels)
        slic_connectivity_pass(self.handle, labels.data_ptr(), out.data_ptr(), _stream_handle(stream))
        return out

    @property
    def launches(self) -> int:
        return slic_launch_count(self.handle)

    @property
    def iterations_run(self) -> int:
        """Centre updates the last run performed (fewer than ``iterations``
        when the stopping test ended it; waits for the device)."""
        return slic_iterations_run(self.handle)


class BatchSegmenter:
    """Many frames (uneven size, S or K, m) segmented by one set of launches
    per pass. ``frames`` is a sequence of dicts with keys width, height and
    K or S, optionally m, color_space, in_channels, perturb_seeds and
    convergence (per frame: a converged frame skips its remaining middle
    passes); ``iterations`` and ``enforce_connectivity`` are shared. Output
    tensors are allocated here (``labels[f]`` int32 [H, W], ``centres[f]``
    float32 [K_eff, 6])."""

    def __init__(self, frames, *, iterations: int = 5, enforce_connectivity: int = 1, device=None):
        import torch
        self.params = [slic_params(f["width"], f["height"], f.get("K", 0), f.get("S", 0), float(f.get("m", 10.0)),
                                   iterations, f.get("color_space", SLIC_CIELAB), int(enforce_connectivity),
                                   f.get("in_channels", 3), int(bool(f.get("perturb_seeds", False))),
                                   float(f.get("convergence", 0.0))) for f in frames]
        self.handle = slic_batch_create(self.params)
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.K_eff = []
        for f in range(len(self.params)):
            _, ns_c, ns_r = slic_batch_grid(self.handle, f)
            self.K_eff.append(ns_c * ns_r)
        # one allocation each for all frames' labels and centres, frame after
        # frame, so that host copies of the whole batch are single copies
        px = [p.height * p.width for p in self.params]
        self._labels_flat = torch.empty(sum(px), dtype=torch.int32, device=dev)
        self._centres_flat = torch.empty(6 * sum(self.K_eff), dtype=torch.float32, device=dev)
        self.labels, self.centres = [], []
        lo = co = 0
        for p, n, k in zip(self.params, px, self.K_eff):
            self.labels.append(self._labels_flat[lo:lo + n].view(p.height, p.width))
            self.centres.append(self._centres_flat[co:co + 6 * k].view(k, 6))
            lo += n
            co += 6 * k
        self.images = None

    def bind(self, images, init_centres=None, stream=None):
        """Bind input tensors (uint8 [H, W, C] CUDA, one per frame); keep them
        alive while in use. The first binding waits for the device; later
        ones are ordered on `stream` (the current stream by default) and do
        not wait (slic_batch_rebind)."""
        for img, p in zip(images, self.params):
            if not img.is_cuda or not img.is_contiguous() or tuple(img.shape) != (p.height, p.width, p.in_channels):
                raise ValueError("each image must be a contiguous uint8 CUDA tensor of its frame's shape")
        first = self.images is None
        self.images = list(images)
        init = None
        if init_centres is not None:
            init = [t.data_ptr() if t is not None else None for t in init_centres]
        args = ([t.data_ptr() for t in self.images], [t.data_ptr() for t in self.labels],
                [t.data_ptr() for t in self.centres], init)
        if first:
            slic_batch_set_buffers(self.handle, *args)
        else:
            self._init_refs = init_centres  # (kept alive until the next binding)
            slic_batch_rebind(self.handle, *args, _stream_handle(stream))

    def segment(self, stream=None):
        slic_batch_segment(self.handle, _stream_handle(stream))
        return self.labels, self.centres

    def set_warmstart(self, net):
        """Arm the learned warm start with a network (an object with a
        ``handle``, e.g. warmstart.WarmStartNet, or a raw slic_net handle),
        or disarm it with None. The network must outlive the arming."""
        self._net = net
        slic_batch_set_warmstart(self.handle, getattr(net, "handle", net) if net is not None else None)

    def segment_host(self, host_images, host_labels=None, host_centres=None, stream=None):
        """End to end with host tensors (page-locked CPU tensors, one per
        frame): images in, labels [H, W] int32 and centres [K_eff, 6] float32
        out (either list, or an entry of it, may be None: that copy is
        skipped). Enqueued on `stream`; synchronise it before reading the
        outputs."""
        ptrs = lambda ts: [t.data_ptr() if t is not None else None for t in ts] if ts is not None else None  # noqa: E731
        slic_batch_segment_host(self.handle, ptrs(host_images), ptrs(host_labels), ptrs(host_centres),
                                _stream_handle(stream))

    def autotune(self, cache_path=None, stream=None):
        """Time the launch shapes that fit; -> (ctas_per_sm, stages, rows, tile_h, fused, groups) chosen."""
        return slic_batch_autotune(self.handle, cache_path, _stream_handle(stream))

    def set_tuning(self, ctas_per_sm: int, stages: int = 0, rows: int = 0, tile_h: int = 0, fused=None,
                   groups=None):
        """A launch shape (as autotune returns it); fused / groups None keep
        those settings."""
        slic_batch_set_tuning(self.handle, ctas_per_sm, stages, rows, tile_h)
        if fused is not None:
            slic_batch_set_fused(self.handle, bool(fused))
        if groups is not None:
            slic_batch_set_groups(self.handle, int(groups))

    def set_groups(self, groups: int):
        """Run the frames as `groups` runs of consecutive frames on
        concurrent streams (1 .. min(4, frames))."""
        slic_batch_set_groups(self.handle, groups)

    def set_fused(self, enable: bool = True):
        """The passes before the last and their updates in one cooperative
        launch, or one launch each (the default)."""
        slic_batch_set_fused(self.handle, enable)

    @property
    def info(self):
        return slic_batch_info(self.handle)

    def status(self):
        """Raises SlicError(SLIC_ERR_TIMEOUT) if a bounded device wait gave up."""
        slic_batch_status(self.handle)

    @property
    def iterations_run(self):
        """Per frame, the centre updates of the last run (waits for the device)."""
        return slic_batch_iterations_run(self.handle, len(self.params))

    def close(self):
        if getattr(self, "handle", None):
            slic_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""ctypes binding of libslicgb.so (include/slic.h), argument marshalling only.

Every function keeps its C name and takes plain integers for device
pointers and streams (e.g. ``tensor.data_ptr()`` and
``torch.cuda.current_stream().cuda_stream``). A non-zero status raises
:class:`SlicError` carrying ``slic_last_error``. The library is loaded on
first use; if it has not been built this raises instead of falling back to
anything else.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

SLIC_OK, SLIC_ERR_INVALID, SLIC_ERR_NOMEM, SLIC_ERR_CUDA, SLIC_ERR_TIMEOUT, SLIC_ERR_STATE = 0, -1, -2, -3, -4, -5
SLIC_CIELAB, SLIC_RGB, SLIC_XYZ = 0, 1, 2
SLIC_FAULT_ALLOC, SLIC_FAULT_WALK_LIMIT, SLIC_FAULT_ABORT_COPIES = 1, 2, 3

_STATUS_NAMES = {0: "SLIC_OK", -1: "SLIC_ERR_INVALID", -2: "SLIC_ERR_NOMEM", -3: "SLIC_ERR_CUDA",
                 -4: "SLIC_ERR_TIMEOUT", -5: "SLIC_ERR_STATE"}


class SlicError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class slic_params(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int), ("K", ctypes.c_int), ("S", ctypes.c_int),
                ("m", ctypes.c_float), ("iterations", ctypes.c_int), ("color_space", ctypes.c_int),
                ("enforce_connectivity", ctypes.c_int), ("in_channels", ctypes.c_int),
                ("perturb_seeds", ctypes.c_int), ("convergence", ctypes.c_float)]


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int

# name -> argtypes (all return slic_status, except slic_last_error)
_SIGNATURES = {
    "slic_create": [ctypes.POINTER(slic_params), ctypes.POINTER(_P)],
    "slic_destroy": [_P],
    "slic_grid": [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "slic_segment": [_P, _P, _P, _P, _P],
    "slic_set_init_centres": [_P, _P],
    "slic_convert": [_P, _P, _P, _P],
    "slic_init_centres": [_P, _P, _P, _P],
    "slic_assign": [_P, _P, _P, _P, _P],
    "slic_update": [_P, _P, _P, _P, _P, _P],
    "slic_connectivity_pass": [_P, _P, _P, _P],
    "slic_launch_count": [_P, ctypes.POINTER(ctypes.c_longlong)],
    "slic_profile_enable": [_P, _I],
    "slic_profile_read": [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)],
    "slic_segment_noalloc": [ctypes.POINTER(slic_params), _P, _P, _P, _P],
    "slic_batch_create": [ctypes.POINTER(slic_params), _I, ctypes.POINTER(_P)],
    "slic_batch_set_buffers": [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P)],
    "slic_batch_rebind": [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P), _P],
    "slic_batch_segment": [_P, _P],
    "slic_batch_segment_host": [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P), _P],
    "slic_batch_set_tuning": [_P, _I, _I, _I, _I],
    "slic_batch_set_fused": [_P, _I],
    "slic_batch_set_groups": [_P, _I],
    "slic_batch_autotune": [_P, ctypes.c_char_p, _P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                            ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "slic_batch_info": [_P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                        ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                        ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "slic_batch_destroy": [_P],
    "slic_batch_status": [_P],
    "slic_batch_iterations_run": [_P, ctypes.POINTER(_I)],
    "slic_iterations_run": [_P, ctypes.POINTER(_I)],
    "slic_connectivity_components": [_P, _P, _P, _P],
    "slic_status_check": [_P],
    "slic_batch_profile_enable": [_P, _I],
    "slic_batch_profile_read": [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)],
    "slic_batch_profile_times": [_P, ctypes.POINTER(ctypes.c_double), _I, ctypes.POINTER(_I)],
    "slic_net_create": [_I, _I, _I, _I, ctypes.c_float, ctypes.c_ulonglong, ctypes.POINTER(_P)],
    "slic_net_destroy": [_P],
    "slic_net_param_count": [_P, ctypes.POINTER(ctypes.c_size_t)],
    "slic_net_get_params": [_P, _I, _P, ctypes.c_size_t],
    "slic_net_set_params": [_P, _P, ctypes.c_size_t],
    "slic_net_forward": [_P, _I, _P, _P, _P, _P],
    "slic_net_gradients": [_P, _I, _P, _P, _P, _P],
    "slic_net_train_step": [_P, _I, _P, _P, ctypes.c_float, _P, _P],
    "slic_net_status": [_P],
    "slic_net_slots": [_P, _I, _P, _P, _P, _P],
    "slic_set_warmstart": [_P, _P],
    "slic_batch_set_warmstart": [_P, _P],
    "slic_batch_grid": [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "slic_noalloc_status_check": [],
    "slic_fault_inject": [_I, ctypes.c_longlong],
}


def library_path() -> str:
    return _build.SLIC_LIB


def lib():
    """Load libslicgb.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_1509_04232_gb300.build.build_all() "
                               "(the CUDA path has no CPU fallback)")
        L = ctypes.CDLL(path)
        for name, args in _SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.slic_last_error.argtypes = [_P]
        L.slic_last_error.restype = ctypes.c_char_p
        L.slic_batch_last_error.argtypes = [_P]
        L.slic_batch_last_error.restype = ctypes.c_char_p
        L.slic_net_last_error.argtypes = [_P]
        L.slic_net_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def slic_last_error(h) -> str:
    return lib().slic_last_error(h).decode()


def _check(status: int, h):
    if status != SLIC_OK:
        raise SlicError(status, slic_last_error(h))


def slic_create(params: slic_params) -> int:
    h = _P()
    _check(lib().slic_create(ctypes.byref(params), ctypes.byref(h)), None)
    return h.value


def slic_destroy(h: int) -> None:
    _check(lib().slic_destroy(h), None)


def slic_grid(h: int):
    s, c, r = _I(), _I(), _I()
    _check(lib().slic_grid(h, ctypes.byref(s), ctypes.byref(c), ctypes.byref(r)), h)
    return s.value, c.value, r.value


def slic_segment(h: int, d_image: int, d_labels: int, d_centres: int, stream: int = 0) -> None:
    _check(lib().slic_segment(h, d_image, d_labels, d_centres, stream or None), h)


def slic_set_init_centres(h: int, d_init: int | None) -> None:
    _check(lib().slic_set_init_centres(h, d_init or None), h)


def slic_set_warmstart(h: int, net: int | None) -> None:
    """Arm (or, with None, disarm) the learned warm start of the handle."""
    _check(lib().slic_set_warmstart(h, net or None), h)


def slic_convert(h: int, d_image: int, d_features: int, stream: int = 0) -> None:
    _check(lib().slic_convert(h, d_image, d_features, stream or None), h)


def slic_init_centres(h: int, d_features: int, d_centres: int, stream: int = 0) -> None:
    _check(lib().slic_init_centres(h, d_features, d_centres, stream or None), h)


def slic_assign(h: int, d_features: int, d_centres: int, d_labels: int, stream: int = 0) -> None:
    _check(lib().slic_assign(h, d_features, d_centres, d_labels, stream or None), h)


def slic_update(h: int, d_features: int, d_labels: int, d_centres_in: int, d_centres_out: int,
                stream: int = 0) -> None:
    _check(lib().slic_update(h, d_features, d_labels, d_centres_in, d_centres_out, stream or None), h)


def slic_connectivity_pass(h: int, d_in: int, d_out: int, stream: int = 0) -> None:
    _check(lib().slic_connectivity_pass(h, d_in, d_out, stream or None), h)


def slic_launch_count(h: int) -> int:
    n = ctypes.c_longlong()
    _check(lib().slic_launch_count(h, ctypes.byref(n)), h)
    return n.value


def slic_profile_enable(h: int, enable: bool) -> None:
    _check(lib().slic_profile_enable(h, int(bool(enable))), h)


def slic_profile_read(h: int):
    ms, n = ctypes.c_double(), ctypes.c_longlong()
    _check(lib().slic_profile_read(h, ctypes.byref(ms), ctypes.byref(n)), h)
    return ms.value, n.value


def slic_segment_noalloc(params: slic_params, d_image: int, d_labels: int, d_centres: int, stream: int = 0) -> None:
    """Whole segmentation without any device allocation (scratch in a static
    32 MiB device array shared by all calls; see include/slic.h)."""
    _check(lib().slic_segment_noalloc(ctypes.byref(params), d_image, d_labels, d_centres, stream or None), None)


def slic_noalloc_status_check() -> None:
    """Raise SlicError(SLIC_ERR_TIMEOUT) if a bounded loop of the
    allocation-free path gave up since the last check (waits for the device)."""
    _check(lib().slic_noalloc_status_check(), None)


def slic_fault_inject(kind: int, value: int) -> None:
    """Fault injection for tests of failure detection (include/slic.h)."""
    _check(lib().slic_fault_inject(int(kind), int(value)), None)


# --- batches ---------------------------------------------------------------

def slic_batch_last_error(b) -> str:
    return lib().slic_batch_last_error(b).decode()


def _bcheck(status: int, b):
    if status != SLIC_OK:
        raise SlicError(status, slic_batch_last_error(b))


def _ptr_array(ptrs):
    return (_P * len(ptrs))(*[p or None for p in ptrs])


def slic_batch_create(params) -> int:
    """params: sequence of slic_params, one per frame."""
    arr = (slic_params * len(params))(*params)
    b = _P()
    _bcheck(lib().slic_batch_create(arr, len(params), ctypes.byref(b)), None)
    return b.value


def slic_batch_set_buffers(b: int, d_images, d_labels, d_centres, d_init=None) -> None:
    init = _ptr_array(d_init) if d_init is not None else None
    _bcheck(lib().slic_batch_set_buffers(b, _ptr_array(d_images), _ptr_array(d_labels), _ptr_array(d_centres),
                                         init), b)


def slic_batch_rebind(b: int, d_images, d_labels, d_centres, d_init=None, stream: int = 0) -> None:
    """Stream-ordered rebinding (no device-wide wait); see include/slic.h."""
    init = _ptr_array(d_init) if d_init is not None else None
    _bcheck(lib().slic_batch_rebind(b, _ptr_array(d_images), _ptr_array(d_labels), _ptr_array(d_centres), init,
                                    stream or None), b)


def slic_batch_segment(b: int, stream: int = 0) -> None:
    _bcheck(lib().slic_batch_segment(b, stream or None), b)


def slic_batch_segment_host(b: int, host_images, host_labels=None, host_centres=None, stream: int = 0) -> None:
    """host_* are sequences of host addresses (page-locked memory), one per frame."""
    n = len(host_images)

    def arr(ptrs):
        return (_P * n)(*[p or None for p in ptrs]) if ptrs is not None else None

    _bcheck(lib().slic_batch_segment_host(b, arr(host_images), arr(host_labels), arr(host_centres),
                                          stream or None), b)


def slic_batch_set_tuning(b: int, ctas_per_sm: int, stages: int = 0, rows: int = 0, tile_h: int = 0) -> None:
    _bcheck(lib().slic_batch_set_tuning(b, int(ctas_per_sm), int(stages), int(rows), int(tile_h)), b)


def slic_batch_set_fused(b: int, enable: bool) -> None:
    _bcheck(lib().slic_batch_set_fused(b, 1 if enable else 0), b)


def slic_batch_set_groups(b: int, groups: int) -> None:
    _bcheck(lib().slic_batch_set_groups(b, int(groups)), b)


def slic_batch_autotune(b: int, cache_path: str | None = None, stream: int = 0):
    """-> (ctas_per_sm, stages, rows, tile_h, fused, groups) chosen."""
    c, st, rw, th, fu, gr = _I(), _I(), _I(), _I(), _I(), _I()
    path = cache_path.encode() if cache_path else None
    _bcheck(lib().slic_batch_autotune(b, path, stream or None, ctypes.byref(c), ctypes.byref(st), ctypes.byref(rw),
                                      ctypes.byref(th), ctypes.byref(fu), ctypes.byref(gr)), b)
    return c.value, st.value, rw.value, th.value, fu.value, gr.value


def slic_batch_info(b: int):
    """-> (total_pixels, launches, ctas_per_sm, stages, rows, tile_h, fused, groups)."""
    px, n, c, st, rw, th, fu, gr = ctypes.c_longlong(), ctypes.c_longlong(), _I(), _I(), _I(), _I(), _I(), _I()
    _bcheck(lib().slic_batch_info(b, ctypes.byref(px), ctypes.byref(n), ctypes.byref(c), ctypes.byref(st),
                                  ctypes.byref(rw), ctypes.byref(th), ctypes.byref(fu), ctypes.byref(gr)), b)
    return px.value, n.value, c.value, st.value, rw.value, th.value, fu.value, gr.value


def slic_connectivity_components(h: int, d_in: int, d_out: int, stream: int = 0) -> None:
    _check(lib().slic_connectivity_components(h, d_in, d_out, stream or None), h)


def slic_status_check(h: int) -> None:
    """Raise SlicError(SLIC_ERR_TIMEOUT) if a bounded device loop gave up."""
    _check(lib().slic_status_check(h), h)


def slic_iterations_run(h: int) -> int:
    """Centre updates performed by the handle's last run (waits for the device)."""
    n = _I()
    _check(lib().slic_iterations_run(h, ctypes.byref(n)), h)
    return n.value


def slic_batch_iterations_run(b: int, n_frames: int) -> list:
    """Centre updates each frame's last run performed (waits for the device)."""
    out = (_I * n_frames)()
    _bcheck(lib().slic_batch_iterations_run(b, out), b)
    return list(out)


def slic_batch_status(b: int) -> None:
    """Raise SlicError(SLIC_ERR_TIMEOUT) if a bounded device wait gave up."""
    _bcheck(lib().slic_batch_status(b), b)


def slic_batch_profile_enable(b: int, enable: bool) -> None:
    _bcheck(lib().slic_batch_profile_enable(b, int(bool(enable))), b)


def slic_batch_profile_read(b: int):
    ms, n = ctypes.c_double(), ctypes.c_longlong()
    _bcheck(lib().slic_batch_profile_read(b, ctypes.byref(ms), ctypes.byref(n)), b)
    return ms.value, n.value


def slic_batch_profile_times(b: int, max_n: int = 4096):
    buf = (ctypes.c_double * max_n)()
    n = _I()
    _bcheck(lib().slic_batch_profile_times(b, buf, max_n, ctypes.byref(n)), b)
    return list(buf[:n.value])


def slic_batch_grid(b: int, frame: int):
    """-> (S, ns_c, ns_r) of one frame of the batch."""
    s, c, r = _I(), _I(), _I()
    _bcheck(lib().slic_batch_grid(b, int(frame), ctypes.byref(s), ctypes.byref(c), ctypes.byref(r)), b)
    return s.value, c.value, r.value


def slic_batch_set_warmstart(b: int, net: int | None) -> None:
    """Arm (or, with None, disarm) the learned warm start of every frame."""
    _bcheck(lib().slic_batch_set_warmstart(b, net or None), b)


def slic_batch_destroy(b: int) -> None:
    _bcheck(lib().slic_batch_destroy(b), None)


# --- learned warm start network ----------------------------------------------

def slic_net_last_error(n) -> str:
    return lib().slic_net_last_error(n).decode()


def _ncheck(status: int, n):
    if status != SLIC_OK:
        raise SlicError(status, slic_net_last_error(n))


def slic_net_create(max_batch: int, width: int, height: int, S: int, m: float = 10.0, seed: int = 0) -> int:
    n = _P()
    _ncheck(lib().slic_net_create(max_batch, width, height, S, float(m), seed, ctypes.byref(n)), None)
    return n.value


def slic_net_destroy(n: int) -> None:
    _ncheck(lib().slic_net_destroy(n), None)


def slic_net_param_count(n: int) -> int:
    c = ctypes.c_size_t()
    _ncheck(lib().slic_net_param_count(n, ctypes.byref(c)), n)
    return c.value


def slic_net_get_params(n: int, which: int = 0):
    import numpy as np
    out = np.empty(slic_net_param_count(n), np.float32)
    _ncheck(lib().slic_net_get_params(n, which, out.ctypes.data_as(_P), out.size), n)
    return out


def slic_net_set_params(n: int, params) -> None:
    import numpy as np
    arr = np.ascontiguousarray(params, dtype=np.float32)
    _ncheck(lib().slic_net_set_params(n, arr.ctypes.data_as(_P), arr.size), n)


def slic_net_forward(n: int, batch: int, d_images: int, d_logits: int | None, d_labels: int | None,
                     stream: int = 0) -> None:
    _ncheck(lib().slic_net_forward(n, batch, d_images, d_logits or None, d_labels or None, stream or None), n)


def slic_net_gradients(n: int, batch: int, d_images: int, d_targets: int, d_stats: int | None,
                       stream: int = 0) -> None:
    _ncheck(lib().slic_net_gradients(n, batch, d_images, d_targets, d_stats or None, stream or None), n)


def slic_net_status(n: int) -> None:
    """Raises SlicError(SLIC_ERR_TIMEOUT) if a bounded device wait of the network gave up."""
    _ncheck(lib().slic_net_status(n), n)


def slic_net_train_step(n: int, batch: int, d_images: int, d_targets: int, lr: float, d_stats: int | None,
                        stream: int = 0) -> None:
    _ncheck(lib().slic_net_train_step(n, batch, d_images, d_targets, float(lr), d_stats or None, stream or None), n)


def slic_net_slots(n: int, batch: int, d_labels: int, d_slots: int, d_bad: int | None, stream: int = 0) -> None:
    _ncheck(lib().slic_net_slots(n, batch, d_labels, d_slots, d_bad or None, stream or None), n)

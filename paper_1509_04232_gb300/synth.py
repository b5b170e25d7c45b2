"""Seeded synthetic inputs: Voronoi colour images and videos.

Inputs only -- none of SLIC's arithmetic lives here, so the CUDA path, the
FP64 oracle's tests and the benchmark all read identical bytes from this
module. The renderer is ``csrc/synth.c`` (counter-based SplitMix64 draws,
Box-Muller normals, round half to even), compiled by ``build.build_synth``.

Workload recipes (image sizes, region counts, noise levels) follow the
evaluation settings this library is benchmarked on: a 320x240 image with 40
regions and noise sigma 8; 1920x1080 with 400 regions and sigma 6 (plus
640x480); a 256-frame batch of mixed resolutions; 256x256 training images;
a 3840x2160 video whose regions move 0-4 px/frame with colour drift sigma 2.
Seeds are ``workload_id * 2**32 + frame_index``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


class _Spec(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int), ("channels", ctypes.c_int),
                ("regions", ctypes.c_int), ("noise_sigma", ctypes.c_double),
                ("grad_max", ctypes.c_double), ("vmax", ctypes.c_double),
                ("drift_sigma", ctypes.c_double), ("seed", ctypes.c_uint64)]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build_synth())
        lib.synth_frame.argtypes = [ctypes.POINTER(_Spec), ctypes.c_int, ctypes.c_void_p]
        lib.synth_frame.restype = ctypes.c_int
        _lib = lib
    return _lib


def voronoi_frame(width: int, height: int, regions: int, sigma: float, seed: int, *,
                  grad_max: float = 30.0, channels: int = 3, t: int = 0, vmax: float = 0.0,
                  drift_sigma: float = 0.0, out: np.ndarray | None = None) -> np.ndarray:
    """Render one uint8 [H, W, channels] frame (frame ``t`` of a video when
    ``vmax``/``drift_sigma`` are non-zero)."""
    spec = _Spec(width, height, channels, regions, float(sigma), float(grad_max), float(vmax),
                 float(drift_sigma), int(seed) & 0xFFFFFFFFFFFFFFFF)
    if out is None:
        out = np.empty((height, width, channels), np.uint8)
    assert out.shape == (height, width, channels) and out.dtype == np.uint8 and out.flags.c_contiguous
    rc = _load().synth_frame(ctypes.byref(spec), int(t), out.ctypes.data_as(ctypes.c_void_p))
    if rc != 0:
        raise ValueError(f"synth_frame failed with status {rc}")
    return out


def seed_of(workload_id: int, frame: int) -> int:
    return (int(workload_id) << 32) + int(frame)


# --- workload recipes -------------------------------------------------------

def small_image(frame: int = 0) -> np.ndarray:
    """320x240, 40 regions, noise sigma 8 (parity workload; K=300, m=10, 10 it)."""
    return voronoi_frame(320, 240, 40, 8.0, seed_of(0, frame))


def hd_image(frame: int = 0, width: int = 1920, height: int = 1080) -> np.ndarray:
    """1920x1080 (or 640x480), 400 regions, noise sigma 6 (S=16, m=10, 5 it)."""
    return voronoi_frame(width, height, 400, 6.0, seed_of(1, frame))


MIXED_SIZES = ((640, 480), (1280, 720), (1920, 1080), (3840, 2160))


def mixed_batch_specs(n_frames: int = 256, seed: int = 2):
    """Per-frame (width, height, S, m) for the mixed-resolution batch: equal
    shares of the four sizes, S drawn from {8,16,32} and m from {5,10,20}
    with a seeded draw."""
    rng = np.random.Generator(np.random.PCG64(seed))
    specs = []
    for f in range(n_frames):
        w, h = MIXED_SIZES[(f * len(MIXED_SIZES)) // n_frames]
        S = int(rng.choice([8, 16, 32]))
        m = float(rng.choice([5.0, 10.0, 20.0]))
        specs.append((w, h, S, m))
    return specs


def mixed_batch_frame(f: int, width: int, height: int) -> np.ndarray:
    return voronoi_frame(width, height, 400, 6.0, seed_of(2, f))


def train_image(index: int) -> np.ndarray:
    """256x256 training image for the learned warm start (seeds 0..)."""
    return voronoi_frame(256, 256, 40, 6.0, seed_of(3, index))


def video_frame(t: int, width: int = 3840, height: int = 2160) -> np.ndarray:
    """Frame t of the 3840x2160 video: 400 regions moving 0-4 px/frame,
    colour drift sigma 2 per frame, noise sigma 6."""
    return voronoi_frame(width, height, 400, 6.0, seed_of(4, 0), t=t, vmax=4.0, drift_sigma=2.0)

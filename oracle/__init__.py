"""FP64 CPU oracle for SLIC superpixels (gSLICr, arXiv 1509.04232).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / reference legs are the only callers. The
product path (the CUDA library and its binding) never imports this package.

The arithmetic lives in ``slic_oracle.c`` (plain C, double precision, the
paper's steps in the paper's order); this module compiles it with gcc and
marshals numpy arrays through ctypes. Function-level citations:

=====================  ==========================================================
``grid``               Sec. 2, S = sqrt(N/K); integer S, ceil grid
``convert``            Sec. 2 (CIELAB) and Sec. 3 "Image space conversion"
``init_centres``       Sec. 3 "Cluster center initialisation"
``perturb_seeds``      Sec. 2, centres moved to the lowest-gradient pixel nearby
``residual``           Sec. 2, L1 change of the centres (the stopping test)
``assign``             Eq. (1) and Sec. 3 "Finding the cluster associations"
``update``             Sec. 3 "Updating the cluster center"
``connectivity_pass``  Sec. 3 "Enforce connectivity" (one of the two passes)
``connectivity_components``  Sec. 2, the original SLIC's component-based connectivity
``slic``               Sec. 4, the Perform_Segmentation stage order
=====================  ==========================================================
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "slic_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

CIELAB, RGB, XYZ = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile ``slic_oracle.c`` into ``liboracle.so`` (no FMA contraction,
    no fast-math, so x86 and Arm give the same doubles)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(cmd, check=True, capture_output=True, text=True)
        os.replace(tmp, _LIB_PATH)
    except subprocess.CalledProcessError as e:
        os.unlink(tmp)
        raise RuntimeError(f"oracle build failed: {e.stderr}") from e
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        lib.oracle_grid.argtypes = [I, I, I, I, P, P, P]
        lib.oracle_convert.argtypes = [P, I, I, I, I, P]
        lib.oracle_init_centres.argtypes = [P, I, I, I, P]
        lib.oracle_assign.argtypes = [P, I, I, I, D, P, P, P]
        lib.oracle_update.argtypes = [P, I, I, P, I, P]
        lib.oracle_connectivity_pass.argtypes = [P, I, I, P]
        lib.oracle_slic.argtypes = [P, I, I, I, I, I, D, I, I, I, P, I, D, P, P, P, P, P]
        lib.oracle_perturb_seeds.argtypes = [P, I, I, I, P, P, P]
        lib.oracle_connectivity_components.argtypes = [P, I, I, I, P]
        lib.oracle_connectivity_components.restype = I
        lib.oracle_residual.argtypes = [P, P, I]
        lib.oracle_residual.restype = D
        for f in (lib.oracle_grid, lib.oracle_convert, lib.oracle_init_centres, lib.oracle_assign,
                  lib.oracle_update, lib.oracle_connectivity_pass, lib.oracle_slic, lib.oracle_perturb_seeds):
            f.restype = I
        _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


def grid(W: int, H: int, K: int = 0, S: int = 0):
    """Return (S, ns_c, ns_r); K_eff = ns_c * ns_r."""
    s, c, r = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(_load().oracle_grid(W, H, K, S, ctypes.byref(s), ctypes.byref(c), ctypes.byref(r)), "grid")
    return s.value, c.value, r.value


def convert(rgb: np.ndarray, color_space: int = CIELAB) -> np.ndarray:
    """uint8 [H,W,3|4] -> float64 [H,W,3] features (L,a,b by default)."""
    rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
    H, W, C = rgb.shape
    out = np.empty((H, W, 3), np.float64)
    _check(_load().oracle_convert(_ptr(rgb), W, H, C, color_space, _ptr(out)), "convert")
    return out


def init_centres(feat: np.ndarray, S: int) -> np.ndarray:
    """float64 [H,W,3] -> centres float64 [K_eff,6] = (l,a,b,x,y,count)."""
    feat = np.ascontiguousarray(feat, dtype=np.float64)
    H, W, _ = feat.shape
    K_eff = -(-W // S) * -(-H // S)
    out = np.empty((K_eff, 6), np.float64)
    _check(_load().oracle_init_centres(_ptr(feat), W, H, S, _ptr(out)), "init_centres")
    return out


def perturb_seeds(feat: np.ndarray, S: int, centres: np.ndarray):
    """Seed perturbation of grid-initialised centres. Returns (centres,
    g_best [K_eff], margin [K_eff]): the gradient at each chosen pixel and
    the relative gap to the next-lowest candidate."""
    feat = np.ascontiguousarray(feat, dtype=np.float64)
    out = np.array(centres, dtype=np.float64, copy=True, order="C")
    H, W, _ = feat.shape
    g = np.empty(out.shape[0], np.float64)
    mg = np.empty(out.shape[0], np.float64)
    _check(_load().oracle_perturb_seeds(_ptr(feat), W, H, S, _ptr(out), _ptr(g), _ptr(mg)), "perturb_seeds")
    return out, g, mg


def residual(prev: np.ndarray, cur: np.ndarray) -> float:
    """Mean L1 move of the centre positions between two centre sets."""
    prev = np.ascontiguousarray(prev, dtype=np.float64)
    cur = np.ascontiguousarray(cur, dtype=np.float64)
    return float(_load().oracle_residual(_ptr(prev), _ptr(cur), prev.shape[0]))


def assign(feat: np.ndarray, S: int, m: float, centres: np.ndarray):
    """One assignment pass. Returns (labels int32 [H,W], margin float64 [H,W])."""
    feat = np.ascontiguousarray(feat, dtype=np.float64)
    centres = np.ascontiguousarray(centres, dtype=np.float64)
    H, W, _ = feat.shape
    labels = np.empty((H, W), np.int32)
    margin = np.empty((H, W), np.float64)
    _check(_load().oracle_assign(_ptr(feat), W, H, S, float(m), _ptr(centres), _ptr(labels),
                                 _ptr(margin)), "assign")
    return labels, margin


def update(feat: np.ndarray, labels: np.ndarray, centres: np.ndarray) -> np.ndarray:
    """One centre update from a label map; returns the new centres."""
    feat = np.ascontiguousarray(feat, dtype=np.float64)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    out = np.array(centres, dtype=np.float64, copy=True, order="C")
    H, W, _ = feat.shape
    _check(_load().oracle_update(_ptr(feat), W, H, _ptr(labels), out.shape[0], _ptr(out)), "update")
    return out


def connectivity_pass(labels: np.ndarray) -> np.ndarray:
    """One connectivity pass (reads the input, returns a new map)."""
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    H, W = labels.shape
    out = np.empty_like(labels)
    _check(_load().oracle_connectivity_pass(_ptr(labels), W, H, _ptr(out)), "connectivity")
    return out


def connectivity_components(labels: np.ndarray, min_size: int):
    """Component-based relabelling (original SLIC's connectivity). Returns
    (new labels int32 [H,W], number of segments kept)."""
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    H, W = labels.shape
    out = np.empty_like(labels)
    n = _load().oracle_connectivity_components(_ptr(labels), W, H, int(min_size), _ptr(out))
    if n < 0:
        raise ValueError("oracle connectivity_components failed")
    return out, n


def slic(rgb: np.ndarray, K: int = 0, S: int = 0, m: float = 10.0, iterations: int = 10,
         color_space: int = CIELAB, enforce_connectivity: int = 1,
         init_centres: np.ndarray | None = None, perturb_seeds: bool = False,
         convergence: float = 0.0) -> dict:
    """Whole SLIC run in the order of the paper's Perform_Segmentation.

    Returns a dict with ``labels`` (after connectivity), ``labels_pre``
    (before it), ``centres`` (the ones the final labels were assigned
    against), ``margin`` (tie margin of the final assignment),
    ``iterations_run`` (updates performed) and the grid.
    """
    rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
    H, W, C = rgb.shape
    s, ns_c, ns_r = grid(W, H, K, S)
    labels = np.empty((H, W), np.int32)
    pre = np.empty((H, W), np.int32)
    margin = np.empty((H, W), np.float64)
    centres = np.empty((ns_c * ns_r, 6), np.float64)
    ic = None
    if init_centres is not None:
        ic = np.ascontiguousarray(init_centres, dtype=np.float64)
        if ic.shape != centres.shape:
            raise ValueError("init_centres has the wrong shape")
    run = ctypes.c_int(0)
    conn = int(enforce_connectivity)  # 0 off, 1 (True) the paper's local rule, 2 components
    _check(_load().oracle_slic(_ptr(rgb), W, H, C, K, S, float(m), iterations, color_space,
                               conn, _ptr(ic), int(bool(perturb_seeds)),
                               float(convergence), _ptr(labels), _ptr(centres), _ptr(pre), _ptr(margin),
                               ctypes.byref(run)), "slic")
    return {"labels": labels, "labels_pre": pre, "centres": centres, "margin": margin,
            "iterations_run": run.value, "S": s, "ns_c": ns_c, "ns_r": ns_r}

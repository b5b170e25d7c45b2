"""In-tree build of the package's native libraries.

* ``libslicgb.so``    -- the CUDA kernels and the C ABI declared in
  ``include/slic.h`` (nvcc, sm_103a only, static cudart, no torch types).
* ``libslicsynth.so`` -- the seeded input generator (gcc, OpenMP).

Both are rebuilt only when a source is newer than the library. Host code is
portable C/C++ (no intrinsics, no -march=native) so the same sources build on
x86_64 and aarch64.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import tempfile

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
SLIC_LIB = os.path.join(PKG, "libslicgb.so")
SYNTH_LIB = os.path.join(PKG, "libslicsynth.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libslicgb.so")


def _stale(target: str, sources) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build_synth(force: bool = False) -> str:
    src = os.path.join(CSRC, "synth.c")
    if force or _stale(SYNTH_LIB, [src]):
        fd, tmp = tempfile.mkstemp(suffix=".so", dir=PKG)
        os.close(fd)
        try:
            _run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                  "-fno-fast-math", src, "-o", tmp, "-lm"])
            os.replace(tmp, SYNTH_LIB)
        finally:
            if os.path.exists(tmp):
                os.unlink(tmp)
    return SYNTH_LIB


def cuda_sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def build_slic(force: bool = False, verbose: bool = False) -> str:
    """Compile every .cu under csrc/ for sm_103a (in parallel) and link them
    into libslicgb.so with a static CUDA runtime."""
    srcs = cuda_sources()
    deps = srcs + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    if not (force or _stale(SLIC_LIB, deps)):
        return SLIC_LIB
    nvcc = _nvcc()
    objdir = tempfile.mkdtemp(prefix="slicgb_build_")
    try:
        flags = ["-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC",
                 "-I", INCLUDE, "-I", CSRC, "-Xptxas", "-v" if verbose else "-O3"]

        def compile_one(src):
            obj = os.path.join(objdir, os.path.basename(src) + ".o")
            out = _run([nvcc, *flags, "-c", src, "-o", obj])
            return obj, out

        with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
            results = list(ex.map(compile_one, srcs))
        if verbose:
            for _, out in results:
                print(out)
        fd, tmp = tempfile.mkstemp(suffix=".so", dir=PKG)
        os.close(fd)
        try:
            _run([nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp,
                  *[o for o, _ in results], "-lpthread", "-ldl", "-lrt"])
            os.replace(tmp, SLIC_LIB)
        finally:
            if os.path.exists(tmp):
                os.unlink(tmp)
    finally:
        shutil.rmtree(objdir, ignore_errors=True)
    return SLIC_LIB


def build_all(force: bool = False, verbose: bool = False):
    return build_slic(force, verbose), build_synth(force)

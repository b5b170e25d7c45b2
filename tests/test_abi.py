"""The C-ABI library builds, loads without a GPU, exports every function that
include/*.h declares, and validates arguments before touching CUDA."""
import ctypes
import glob
import os
import re

import pytest

import paper_1509_04232_gb300 as pkg
from paper_1509_04232_gb300 import _binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(slic_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    build.build_slic()
    return _binding.lib()


def test_header_declares_the_core_calls():
    names = _declared_functions()
    for core in ("slic_create", "slic_segment", "slic_destroy", "slic_grid", "slic_last_error"):
        assert core in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    for n in _declared_functions():
        assert hasattr(_binding, n), n


@pytest.mark.parametrize("kw,msg", [
    (dict(width=0), "width"),
    (dict(height=-3), "width"),
    (dict(K=0, S=0), "S > 0 or K > 0"),
    (dict(m=-1.0), "m must"),
    (dict(iterations=-1), "iterations"),
    (dict(color_space=7), "color_space"),
    (dict(in_channels=2), "in_channels"),
    (dict(enforce_connectivity=3), "enforce_connectivity"),
    (dict(width=1 << 21), "width"),
    (dict(perturb_seeds=2), "perturb_seeds"),
    (dict(convergence=-0.5), "convergence"),
    (dict(convergence=float("inf")), "convergence"),
    (dict(convergence=float("nan")), "convergence"),
])
def test_invalid_params_rejected_without_cuda(lib, kw, msg):
    base = dict(width=64, height=48, K=12, S=0, m=10.0, iterations=3, color_space=0,
                enforce_connectivity=1, in_channels=3)
    base.update(kw)
    p = _binding.slic_params(**base)
    with pytest.raises(pkg.SlicError) as ei:
        pkg.slic_create(p)
    assert ei.value.status == _binding.SLIC_ERR_INVALID
    assert msg in str(ei.value)


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.slic_grid(None, None, None, None) == _binding.SLIC_ERR_INVALID
    assert lib.slic_segment(None, None, None, None, None) == _binding.SLIC_ERR_INVALID
    assert lib.slic_destroy(None) == _binding.SLIC_OK
    assert b"NULL" in lib.slic_last_error(None)


def test_library_has_no_torch_dependency(lib):
    # the boundary is plain C: nothing from libtorch/libc10 may be needed
    import subprocess
    out = subprocess.run(["nm", "-D", "--undefined-only", build.SLIC_LIB], capture_output=True, text=True).stdout
    assert "c10" not in out and "torch" not in out


def test_params_struct_matches_the_header():
    """The ctypes mirror of slic_params has the header's fields, in order and
    with matching C types (a mismatch would shift every later field)."""
    text = open(os.path.join(ROOT, "include", "slic.h")).read()
    body = re.search(r"typedef struct \{(.*?)\} slic_params;", text, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        ctype, names = decl.split(None, 1)
        fields += [(n.strip(), ctype) for n in names.split(",")]
    want = {"int": ctypes.c_int, "float": ctypes.c_float}
    got = [(n, t) for n, t in _binding.slic_params._fields_]
    assert [n for n, _ in fields] == [n for n, _ in got]
    for (n, ctype), (_, t) in zip(fields, got):
        assert want[ctype] is t, n


@pytest.mark.parametrize("second,msg", [
    (dict(iterations=4), "same iterations"),
    (dict(enforce_connectivity=2), "same iterations and connectivity"),
    (dict(convergence=-1.0), "convergence"),
    (dict(perturb_seeds=5), "perturb_seeds"),
    (dict(enforce_connectivity=7), "enforce_connectivity"),
    (dict(width=0), "width"),
])
def test_invalid_batches_rejected_without_cuda(lib, second, msg):
    """Per-frame options may differ within a batch, iterations and the
    connectivity mode may not; every frame is validated before any CUDA call."""
    base = dict(width=64, height=48, K=0, S=16, m=10.0, iterations=3, color_space=0,
                enforce_connectivity=1, in_channels=3)
    other = dict(base)
    other.update(second)
    with pytest.raises(pkg.SlicError) as ei:
        pkg.slic_batch_create([_binding.slic_params(**base), _binding.slic_params(**other)])
    assert ei.value.status == _binding.SLIC_ERR_INVALID
    assert msg in str(ei.value)

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built libslicgb.so")


@pytest.fixture(scope="session")
def golden_dir():
    return GOLDEN


@pytest.fixture(scope="session")
def slic_gpu():
    """The CUDA binding on cuda:0; building it first if needed."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("gpu test collected but no CUDA device is visible")
    from paper_1509_04232_gb300 import build
    build.build_all()
    import paper_1509_04232_gb300 as pkg
    return pkg

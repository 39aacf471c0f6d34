import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
TESTS = os.path.dirname(os.path.abspath(__file__))
if TESTS not in sys.path:
    sys.path.insert(0, TESTS)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


@pytest.fixture(scope="session")
def native_gpu():
    """The built library on a machine with a CUDA device (fails loudly otherwise)."""
    import torch
    from paper_2301_09889_gb300 import build, native
    assert torch.cuda.is_available(), "GPU test run without a CUDA device"
    build.build()
    native.load()
    torch.cuda.init()
    return native

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


def gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def cuda_lib():
    """The built C-ABI library (GPU tests only): fails loudly when missing."""
    if not gpu_available():
        pytest.fail("GPU test collected on a machine without a CUDA device")
    from paper_1703_01506_gb300 import binding
    binding.load()
    return binding

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the compiled library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


def cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def gpu_lib():
    """The compiled CUDA library; GPU tests fail loudly when it is missing."""
    if not cuda_available():
        pytest.fail("GPU test collected on a machine without CUDA: run with -m 'not gpu'")
    import paper_2507_11172_gb300 as r3
    r3.load()
    return r3

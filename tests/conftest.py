import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def gplib():
    """The C-ABI binding, with libgp.so built from the in-tree sources if stale."""
    from paper_2503_00246_gb300 import build
    build.build()
    from paper_2503_00246_gb300 import gp
    return gp


@pytest.fixture(scope="session")
def cuda(gplib):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test selected but no CUDA device is visible")
    torch.cuda.set_device(0)
    return torch

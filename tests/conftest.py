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
def svlib():
    """The C-ABI library, built in-tree on first use (host entry points work without a GPU)."""
    from paper_2604_03816_gb300 import build as B
    B.build()
    from paper_2604_03816_gb300 import sv
    return sv


@pytest.fixture(scope="session")
def gpu(svlib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return svlib

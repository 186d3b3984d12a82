import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a) and the built libkcycle.so")
    config.addinivalue_line("markers", "slow: oracle runs that take tens of seconds on the CPU")


@pytest.fixture(scope="session")
def lib():
    """The C-ABI library through its Python binding; GPU tests only."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_00626_b300 import build
    build.build()
    from paper_2010_00626_b300 import kcycle
    return kcycle

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built extension")
    config.addinivalue_line("markers", "slow: long-running CPU test")

import pytest


@pytest.fixture(scope="session")
def skf():
    """The CUDA library through its Python binding (GPU tests only)."""
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2208_11447_gb300 as pkg
    if not os.path.exists(pkg.LIB_PATH):
        from paper_2208_11447_gb300 import build
        build.build()
    pkg.lib()
    return pkg

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libgaincal.so")


@pytest.fixture(scope="session")
def gpu_lib():
    """Build (if needed) and load the CUDA library; the GPU tests all go through it."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test selected but no CUDA device is visible")
    from paper_1502_06974_gb300 import build, _native
    build.build()
    return _native.lib()

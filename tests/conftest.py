import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300); runs libgpe kernels")


@pytest.fixture(scope="session")
def built_lib():
    """Build libgpe.so if needed (nvcc cross-compiles without a GPU)."""
    from paper_1611_02045_gb300 import build
    return build.build()

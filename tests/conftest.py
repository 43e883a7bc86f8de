import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")


@pytest.fixture(scope="session")
def gpu_lib():
    """The CUDA library's Python binding; the test fails loudly if it cannot be loaded."""
    from paper_2602_11709_gb300 import xrd
    xrd.load()
    return xrd

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
def rimo_lib():
    """The compiled CUDA library, built first (nvcc) when it is missing or older than its
    sources.  Host-only entry points run without a GPU."""
    from paper_2605_26347_gb300 import _build, _lib
    if _lib.LIB_PATH == _build.LIB:  # not when RIMO_LIBRARY selects another build
        _build.build()
    return _lib.load()

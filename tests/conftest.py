import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


@pytest.fixture(scope="session")
def ofa():
    """The ctypes binding, building libofa.so first if it is missing or stale."""
    from paper_2206_12661_gb300 import _build
    _build.build()
    from paper_2206_12661_gb300 import ofa as binding
    return binding

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(autouse=True)
def _debug_build_status_clean(request):
    """Under SMCX_DEBUG=1 (the library's bounds-checking debug build), every
    GPU test must leave no out-of-bounds access recorded."""
    yield
    if os.environ.get("SMCX_DEBUG") == "1" and request.node.get_closest_marker("gpu"):
        from paper_2503_12591_gb300 import smcx
        assert smcx.debug_status() == (0, 0)

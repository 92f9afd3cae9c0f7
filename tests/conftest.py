import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the compiled libmp.so")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(params=["plain", "mirror"])
def oracle_arith(request):
    """Run a test once per oracle arithmetic mode (the mode its oracle calls
    use when they name none): the pins must hold for both."""
    import oracle
    old = oracle.DEFAULT_ARITH
    oracle.DEFAULT_ARITH = request.param
    yield request.param
    oracle.DEFAULT_ARITH = old


def pytest_collection_modifyitems(config, items):
    # CPU-only runs (no GPU visible) skip gpu tests only if they were selected explicitly
    pass

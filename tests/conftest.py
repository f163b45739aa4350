import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the compiled library")
    config.addinivalue_line("markers", "slow: long-running oracle comparison")


@pytest.fixture(scope="session", autouse=True)
def _oracle_threads():
    """The oracle's independent subdomain loops run on every host core (its
    results do not depend on the thread count; test_oracle.py checks that)."""
    import oracle
    oracle.set_threads(os.cpu_count() or 1)
    yield

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def lgf_cache():
    """Session cache of oracle LGF tables keyed by (order, nmax)."""
    from oracle.lgf import lgf_table
    cache = {}

    def get(M, nmax):
        key = (M, nmax)
        if key not in cache:
            cache[key] = lgf_table(M, nmax)
        return cache[key]
    return get

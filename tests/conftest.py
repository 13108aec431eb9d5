import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


_cache = {}


def cached_problem(key, builder):
    if key not in _cache:
        _cache[key] = builder()
    return _cache[key]


@pytest.fixture(scope="session")
def c1():
    import femgen
    return cached_problem("c1", femgen.plain_c1)


@pytest.fixture(scope="session")
def c1_linear():
    import femgen
    return cached_problem("c1_linear", lambda: femgen.plain_c1(rhs="linear"))

import functools
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libssgi.so")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@functools.lru_cache(maxsize=None)
def _workload(name):
    import ssgi_inputs as si
    return getattr(si, name)()


@functools.lru_cache(maxsize=None)
def _lut():
    import oracle as O
    return O.build_lut()


@pytest.fixture(scope="session")
def lut():
    return _lut()


@pytest.fixture(scope="session")
def cfg1():
    return _workload("config1")


@pytest.fixture(scope="session")
def small():
    return _workload("small_case")

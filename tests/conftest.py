import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_addoption(parser):
    # the test of the pins runs them against copies of the oracle with one
    # mistake planted, passing each copy's path here
    parser.addoption("--oracle-lib", default=None,
                     help="load the oracle from this shared library (pin tests only)")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")
    lib = config.getoption("--oracle-lib")
    if lib:
        from oracle import oracle
        oracle.use_library(lib)


GOLDEN = os.path.join(ROOT, "tests", "golden")


def hexf(s):
    """float32 from a hex-float / 'inf' string of a golden fixture."""
    import numpy as np
    if s in ("inf", "+inf"):
        return np.float32(np.inf)
    return np.float32(float.fromhex(s))

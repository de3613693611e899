import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a library)")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def ka_params():
    import oracle
    from paper_2001_07089_gb300 import workloads as wl
    return oracle.Params(wl.KA_EPS, wl.KA_SIG, wl.KA_RC, wl.KA_MASS)

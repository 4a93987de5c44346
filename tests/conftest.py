import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def rel_l2(u, v, ur, vr):
    import numpy as np
    num = np.sum((np.asarray(u) - ur) ** 2 + (np.asarray(v) - vr) ** 2)
    den = np.sum(np.asarray(ur) ** 2 + np.asarray(vr) ** 2)
    return float(np.sqrt(num / den)) if den > 0 else float(np.sqrt(num))


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a library)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def tiny_params():
    import oracle as O
    from paper_2406_06761_gb300 import workload as W
    w = W.WORKLOADS["tiny"]
    return O.params(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)


@pytest.fixture(scope="session")
def small_params():
    """N = 16, two 30-bit limbs, t = 929: small enough for big-integer brute force."""
    import oracle as O
    return O.params(4, 2, 30, 10, 4)

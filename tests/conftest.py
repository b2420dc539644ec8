import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA path through the C ABI)")


EPS64 = 2.0 ** -52
EPS32 = 2.0 ** -23


def fp64_tol(m: int, n: int) -> float:
    """Backward-error / orthogonality bound 10 * n * eps * sqrt(m) in FP64."""
    return 10.0 * max(n, 1) * EPS64 * max(m, 1) ** 0.5


def fp32_tol(m: int, n: int) -> float:
    """The same bound with the FP32 unit roundoff."""
    return 10.0 * max(n, 1) * EPS32 * max(m, 1) ** 0.5


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle

    oracle.build()
    return oracle

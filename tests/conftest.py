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
# Relative error of one FP32 product formed from three BF16 products
# (hi*hi + hi*lo + lo*hi): the dropped lo*lo term and the two split residuals
# are each below 2^-16 of |x y|.
EPS_BF16X3 = 2.0 ** -16
# The same with three TF32 products (11-bit significands): the split itself
# leaves about 2^-21 of |x y|, but the tensor cores' FP32 accumulation sets
# the floor -- measured on this GPU at 1.5e-6 of the sum of |terms| for a
# 512-row leaf, with both splits; 2^-18 covers it by a factor of five and is
# still about 2^-7 below the error of a dropped cross term (2^-11).
EPS_TF32X3 = 2.0 ** -18


def fp64_tol(m: int, n: int) -> float:
    """Backward-error / orthogonality bound 10 * n * eps * sqrt(m) in FP64."""
    return 10.0 * max(n, 1) * EPS64 * max(m, 1) ** 0.5


def fp32_tol(m: int, n: int) -> float:
    """The same bound with the FP32 unit roundoff."""
    return 10.0 * max(n, 1) * EPS32 * max(m, 1) ** 0.5


def caqr_mixed_tol(n: int, eps: float, c: float) -> float:
    """Backward-error bound c * sqrt(n) * eps of a CAQR whose trailing updates
    carry a relative product error eps.  Each of the n/b panel updates adds an
    error of order eps (relative, in the Frobenius norm) to the trailing
    matrix; independent rounding errors add in quadrature (the probabilistic
    analysis of Higham and Mary, 2019), which gives sqrt(n/b) * sqrt(b) * eps
    = sqrt(n) * eps, not n * sqrt(m) * eps."""
    return c * max(n, 1) ** 0.5 * eps


def assert_colwise_close(X, Xo, tol, what="X"):
    """|X_ij - Xo_ij| <= tol * ||Xo(:, j)||_2 for every entry."""
    import numpy as np

    X, Xo = np.asarray(X), np.asarray(Xo)
    scale = np.linalg.norm(Xo, axis=0)
    scale = np.where(scale > 0, scale, 1.0)
    ratio = np.abs(X - Xo) / (tol * scale[None, :])
    i, j = np.unravel_index(np.argmax(ratio), ratio.shape)
    assert ratio[i, j] <= 1.0, f"{what}[{i},{j}]: |diff| = {abs(X[i, j] - Xo[i, j]):.3e} is {ratio[i, j]:.2f} x the bound"


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle

    oracle.build()
    return oracle

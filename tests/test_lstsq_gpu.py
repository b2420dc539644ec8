"""Least squares through TSQR (Section 1) on the GPU, against the CPU oracle.

Both forms: the Q-tree applied to the right-hand sides (tsqr_lstsq) and the
R-only form that factors [A, B] (tsqr_solve_r on R11 \\ R12, residual norms
from R22).  Bound on each solution column (first-order perturbation theory
of least squares, Golub and Van Loan 5.3.8):
    ||x - x_o|| <= c u (kappa + kappa^2 ||r|| / (||A|| ||x_o||)) ||x_o||,
with u = 10 n eps sqrt(m) (the QR bound these tests use throughout) and c = 4;
residual norms within c u ||b||.
"""
import ctypes

import numpy as np
import pytest

from conftest import fp32_tol, fp64_tol
from paper_0808_2664_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_0808_2664_gb300 as tq  # noqa: E402


def dev(A, dtype=torch.float64):
    return tq.as_colmajor(torch.from_numpy(np.asfortranarray(A)).to("cuda", dtype))


def check_solution(A, B, X, rn, Xo, rno, u):
    kappa = np.linalg.cond(A)
    nA = np.linalg.norm(A, 2)
    for c in range(B.shape[1]):
        xo = Xo[:, c]
        bound = 4 * u * (kappa + kappa ** 2 * rno[c] / (nA * np.linalg.norm(xo))) * np.linalg.norm(xo)
        assert np.linalg.norm(X[:, c] - xo) <= bound, (c, np.linalg.norm(X[:, c] - xo), bound)
        assert abs(rn[c] - rno[c]) <= 4 * u * np.linalg.norm(B[:, c]), (c, rn[c], rno[c])


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("m,n,k,h", [(20000, 32, 7, 256), (4096, 64, 16, 0), (1000, 5, 1, 64), (100_000, 16, 40, 0)])
def test_qtree_lstsq_matches_oracle(oracle_mod, dtype, m, n, k, h):
    A = inputs.gaussian(m, n, 800 + n)
    B = inputs.gaussian(m, k, 900 + k)
    if dtype == torch.float32:
        A, B = A.astype(np.float32).astype(np.float64), B.astype(np.float32).astype(np.float64)
    Xo, rno = oracle_mod.lstsq(A, B)
    X, rn = tq.lstsq(dev(A, dtype), dev(B, dtype), leaf_rows=h)
    u = (fp64_tol if dtype == torch.float64 else fp32_tol)(m, n)
    check_solution(A, B, X.double().cpu().numpy(), rn.double().cpu().numpy(), Xo, rno, u)


@pytest.mark.parametrize("m,n,k", [(20000, 32, 7), (5000, 50, 14), (300, 3, 1)])
def test_adjoined_r_only_lstsq_matches_oracle(oracle_mod, m, n, k):
    A = inputs.gaussian(m, n, 810 + n)
    B = inputs.gaussian(m, k, 910 + k)
    Xo, rno = oracle_mod.lstsq(A, B)
    X, rn = tq.lstsq(dev(A), dev(B), adjoined=True)
    check_solution(A, B, X.cpu().numpy(), rn.cpu().numpy(), Xo, rno, fp64_tol(m, n + k))


def test_lstsq_consistent_system_and_bf16x3_apply(oracle_mod):
    """B = A X_true: zero residuals; the tensor-core apply flag gives the solution to the 3xBF16 bound."""
    m, n, k = 8192, 64, 8
    A = inputs.gaussian(m, n, 820).astype(np.float32).astype(np.float64)
    Xt = inputs.gaussian(n, k, 821).astype(np.float32).astype(np.float64)
    B = (A @ Xt).astype(np.float32).astype(np.float64)
    Xo, rno = oracle_mod.lstsq(A, B)
    q = tq.tsqr_q_create(m, n, torch.float32, leaf_rows=512, flags=tq.FLAG_APPLY_BF16X3)
    Ad = dev(A, torch.float32)
    R = q.refactor(Ad)
    X, rn = q.lstsq(R, dev(B, torch.float32))
    assert q.sync_status() == 0
    X = X.double().cpu().numpy()
    kappa = np.linalg.cond(A)
    u = 4 * 2.0 ** -16 + fp32_tol(m, n)
    assert np.abs(X - Xo).max() <= 4 * u * kappa * np.abs(Xo).max()
    assert np.all(rn.double().cpu().numpy() <= 4 * u * np.linalg.norm(B, axis=0))
    q.destroy()


def test_solve_r_and_column_norms():
    n, k = 100, 33
    rng = np.random.default_rng(5)
    R = np.triu(rng.standard_normal((n, n))) + 10 * np.eye(n)
    B = rng.standard_normal((n, k))
    X = tq.solve_r(dev(R), dev(B)).cpu().numpy()
    import scipy.linalg as sl

    Xs = sl.solve_triangular(R, B)  # LAPACK's triangular solve, run as a library
    np.testing.assert_allclose(X, Xs, rtol=1e-12, atol=1e-14)
    C = rng.standard_normal((5000, 9))
    np.testing.assert_allclose(tq.column_norms(dev(C)).cpu().numpy(), np.linalg.norm(C, axis=0), rtol=1e-14)


def test_rank_deficient_reported():
    m, n = 2048, 8
    A = inputs.gaussian(m, n, 830)
    A[:, 5] = 0.0
    with pytest.raises(tq.TsqrError) as ei:
        tq.lstsq(dev(A), dev(inputs.gaussian(m, 2, 831)))
    assert ei.value.code == 4  # a zero diagonal entry of R: TSQR_ERR_NONFINITE


def test_lstsq_argument_errors():
    m, n = 1000, 8
    R, q = tq.tsqr_factor(dev(inputs.gaussian(m, n, 832)))
    L = tq._lib.lib()
    B = dev(inputs.gaussian(m, 2, 833))
    X = tq.colmajor(n, 2, torch.float64)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    vp = ctypes.c_void_p
    assert L.tsqr_lstsq(None, vp(R.data_ptr()), n, 2, vp(B.data_ptr()), m, vp(X.data_ptr()), n, None, s) == 6
    assert L.tsqr_lstsq(q.ptr, vp(R.data_ptr()), n - 1, 2, vp(B.data_ptr()), m, vp(X.data_ptr()), n, None, s) == -3
    assert L.tsqr_lstsq(q.ptr, vp(R.data_ptr()), n, 2, vp(B.data_ptr()), m - 1, vp(X.data_ptr()), n, None, s) == -6
    assert L.tsqr_lstsq(q.ptr, vp(R.data_ptr()), n, 0, None, m, None, n, None, s) == 0
    assert L.tsqr_solve_r(200, 1, 0, vp(R.data_ptr()), 200, vp(X.data_ptr()), 200, None, s) == 5
    q.destroy()

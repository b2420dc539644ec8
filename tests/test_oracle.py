"""Pins for the CPU oracle: facts fixed by the paper and by the mathematics.

Each test checks the oracle against something other than itself: hand-derived
exact factorisations, an exact rational QR, the Cholesky factor of the Gram
matrix, LAPACK run as a library, invariances the paper states, the explicit
product of reflectors, and central finite differences.
"""
import math
import os

import numpy as np
import pytest

from conftest import EPS64, fp64_tol
from paper_0808_2664_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _val(tok: str) -> float:
    return float(eval(tok, {"__builtins__": {}}, {"sqrt": math.sqrt}))


def _load_exact_cases():
    cases, lines = [], [l.strip() for l in open(os.path.join(GOLDEN, "qr_small_exact.txt"))]
    lines = [l for l in lines if l and not l.startswith("#")]
    i = 0
    while i < len(lines):
        _, m, n = lines[i].split()
        m, n = int(m), int(n)
        A = np.array([[_val(t) for t in lines[i + 1 + r].split()] for r in range(m)])
        i += 1 + m
        assert lines[i] == "R"
        R = np.array([[_val(t) for t in lines[i + 1 + r].split()] for r in range(n)])
        i += 1 + n
        assert lines[i] == "Q"
        Q = np.array([[_val(t) for t in lines[i + 1 + r].split()] for r in range(m)])
        i += 1 + m
        cases.append((A, R, Q))
    return cases


@pytest.mark.parametrize("case", range(4))
def test_exact_small_cases(oracle_mod, case):
    A, R_exact, Q_exact = _load_exact_cases()[case]
    Q, R = oracle_mod.qr(A)
    np.testing.assert_allclose(R, R_exact, rtol=0, atol=8 * EPS64 * np.abs(R_exact).max())
    np.testing.assert_allclose(Q, Q_exact, rtol=0, atol=8 * EPS64)


@pytest.mark.parametrize("seed", range(6))
def test_2x2_closed_form(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    a, b, c, d = rng.standard_normal(4)
    A = np.array([[a, b], [c, d]])
    r11 = math.hypot(a, c)
    det = a * d - b * c
    R_cf = np.array([[r11, (a * b + c * d) / r11], [0.0, abs(det) / r11]])
    Q_cf = np.array([[a / r11, -math.copysign(1.0, det) * c / r11],
                     [c / r11, math.copysign(1.0, det) * a / r11]])
    Q, R = oracle_mod.qr(A)
    np.testing.assert_allclose(R, R_cf, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(Q, Q_cf, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("seed", range(4))
def test_3x2_gram_schmidt_closed_form(oracle_mod, seed):
    rng = np.random.default_rng(100 + seed)
    A = rng.standard_normal((3, 2))
    a1, a2 = A[:, 0], A[:, 1]
    r11 = math.sqrt(a1 @ a1)
    q1 = a1 / r11
    r12 = q1 @ a2
    u = a2 - r12 * q1
    r22 = math.sqrt(u @ u)
    Q, R = oracle_mod.qr(A)
    np.testing.assert_allclose(R, [[r11, r12], [0, r22]], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(Q, np.stack([q1, u / r22], axis=1), rtol=1e-12, atol=1e-13)


def test_exact_rational_brute_force(oracle_mod):
    """Exact QR of small integer matrices by sympy (exact Gram-Schmidt)."""
    sympy = pytest.importorskip("sympy")
    rng = np.random.default_rng(7)
    for m, n in ((4, 3), (5, 2), (6, 4)):
        Ai = rng.integers(-9, 10, size=(m, n))
        Qs, Rs = sympy.Matrix(Ai.tolist()).QRdecomposition()
        Q_ex = np.array(Qs.evalf(30).tolist(), dtype=np.float64)
        R_ex = np.array(Rs.evalf(30).tolist(), dtype=np.float64)
        Q, R = oracle_mod.qr(Ai.astype(np.float64))
        np.testing.assert_allclose(R, R_ex, rtol=0, atol=50 * EPS64 * np.abs(R_ex).max())
        np.testing.assert_allclose(Q, Q_ex, rtol=0, atol=50 * EPS64 * n)


@pytest.mark.parametrize("m,n", [(300, 20), (2000, 64), (129, 128)])
def test_gram_cholesky(oracle_mod, m, n):
    """R^T R = A^T A: R is the Cholesky factor of the Gram matrix (well conditioned A)."""
    A = inputs.gaussian(m, n, seed=11 + n)
    _, R = oracle_mod.qr(A, want_q=False)
    L = np.linalg.cholesky(A.T @ A)
    kappa = np.linalg.cond(A)
    err = np.linalg.norm(R - L.T) / np.linalg.norm(L)
    assert err <= fp64_tol(m, n) * kappa, err


@pytest.mark.parametrize("m,n", [(4096, 32), (1000, 7), (64, 64)])
def test_lapack_library_crosscheck(oracle_mod, m, n):
    A = inputs.gaussian(m, n, seed=5)
    Q, R = oracle_mod.qr(A)
    Ql, Rl = np.linalg.qr(A)
    s = np.sign(np.diag(Rl))
    Ql, Rl = Ql * s[None, :], Rl * s[:, None]
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(R - Rl) / np.linalg.norm(Rl) <= fp64_tol(m, n) * kappa
    assert np.linalg.norm(Q - Ql) <= fp64_tol(m, n) * kappa


@pytest.mark.parametrize("kind", ["gaussian", "ill"])
def test_backward_error_and_orthogonality(oracle_mod, kind):
    m, n = 4096, 32
    A = inputs.gaussian(m, n, 1000) if kind == "gaussian" else inputs.ill_conditioned(m, n, 2000)
    Q, R = oracle_mod.qr(A)
    assert np.all(np.diag(R) >= 0)
    assert np.array_equal(R, np.triu(R))
    assert np.linalg.norm(A - Q @ R) / np.linalg.norm(A) <= fp64_tol(m, n)
    assert np.linalg.norm(np.eye(n) - Q.T @ Q) <= fp64_tol(m, n)


def test_row_permutation_invariance(oracle_mod):
    """QR of a row permutation of A has the same R (Section 2.2, model assumptions)."""
    A = inputs.gaussian(777, 16, 3)
    perm = np.random.default_rng(0).permutation(777)
    _, R1 = oracle_mod.qr(A, want_q=False)
    _, R2 = oracle_mod.qr(A[perm], want_q=False)
    assert np.linalg.norm(R1 - R2) / np.linalg.norm(R1) <= fp64_tol(777, 16)


def _tree_r(oracle_mod, blocks, arity):
    rs = [oracle_mod.qr(b, want_q=False)[1] for b in blocks]
    while len(rs) > 1:
        rs = [oracle_mod.qr(np.vstack(rs[i:i + arity]), want_q=False)[1] for i in range(0, len(rs), arity)]
    return rs[0]


def test_tree_shape_invariance(oracle_mod):
    """Binary, arity-4, flat and trivial trees give the same R (Section 2.1, any tree is valid)."""
    m, n, h = 4096, 32, 256
    A = inputs.gaussian(m, n, 1000)
    blocks = [A[i:i + h] for i in range(0, m, h)]
    _, R_triv = oracle_mod.qr(A, want_q=False)
    R_bin = _tree_r(oracle_mod, blocks, 2)
    R_q4 = _tree_r(oracle_mod, blocks, 4)
    R_flat = oracle_mod.qr(blocks[0], want_q=False)[1]
    for b in blocks[1:]:
        R_flat = oracle_mod.qr(np.vstack([R_flat, b]), want_q=False)[1]
    for R in (R_bin, R_q4, R_flat):
        assert np.linalg.norm(R - R_triv) / np.linalg.norm(R_triv) <= fp64_tol(m, n)


def test_stacked_triangles_node(oracle_mod):
    """A tree node: R([Ra; Rb]) = chol(Ra^T Ra + Rb^T Rb)^T (Section 2.1, Eq. TSQR_binarytree_2)."""
    n = 24
    Ra = oracle_mod.qr(inputs.gaussian(100, n, 1), want_q=False)[1]
    Rb = oracle_mod.qr(inputs.gaussian(100, n, 2), want_q=False)[1]
    f = oracle_mod.geqr2(np.vstack([Ra, Rb]))
    L = np.linalg.cholesky(Ra.T @ Ra + Rb.T @ Rb)
    assert np.linalg.norm(f.R - L.T) / np.linalg.norm(L) <= 1e-13
    # Structure: the reflectors of a stacked-triangle node touch row j of the top
    # triangle and rows 0..j of the bottom one, so the bottom half of Y is upper triangular.
    Yb = f.Y[n:, :]
    assert np.array_equal(Yb, np.triu(Yb))


@pytest.mark.parametrize("e", [600, -600])
def test_scaled_inputs_no_overflow(oracle_mod, e):
    A = inputs.gaussian(300, 12, 9)
    s = 2.0 ** e
    _, R = oracle_mod.qr(A, want_q=False)
    _, Rs = oracle_mod.qr(A * s, want_q=False)
    assert np.all(np.isfinite(Rs))
    np.testing.assert_allclose(Rs / s, R, rtol=1e-13, atol=1e-13 * np.abs(R).max())


def test_zero_and_rank_deficient_columns(oracle_mod):
    A = inputs.gaussian(50, 6, 4)
    A[:, 2] = 0.0
    A[:, 4] = A[:, 1] * 3.0
    f = oracle_mod.geqr2(A)
    assert f.tau[2] == 0.0
    Q = oracle_mod.form_q(f)
    R = f.R
    assert np.linalg.norm(A - Q @ R) <= fp64_tol(50, 6) * np.linalg.norm(A)
    assert np.linalg.norm(np.eye(6) - Q.T @ Q) <= fp64_tol(50, 6)
    assert np.all(np.diag(R) >= 0)
    # Degenerate shapes: one column, one row, square.
    for shape in ((1, 1), (9, 1), (5, 5)):
        B = inputs.gaussian(*shape, 12)
        Qb, Rb = oracle_mod.qr(B)
        assert np.allclose(Qb @ Rb, B, atol=1e-14 * max(1, np.abs(B).max()))


def test_apply_qt_gives_r_and_roundtrip(oracle_mod):
    m, n, k = 513, 17, 5
    A = inputs.gaussian(m, n, 21)
    f = oracle_mod.geqr2(A)
    QtA = oracle_mod.apply_qt(f, A)
    np.testing.assert_allclose(QtA[:n], f.R, atol=fp64_tol(m, n) * np.linalg.norm(A))
    assert np.linalg.norm(QtA[n:]) <= fp64_tol(m, n) * np.linalg.norm(A)
    C = inputs.gaussian(m, k, 22)
    back = oracle_mod.apply_q(f, oracle_mod.apply_qt(f, C))
    assert np.linalg.norm(back - C) <= fp64_tol(m, n) * np.linalg.norm(C)
    # apply_q on [I; 0] is the thin Q.
    E = np.zeros((m, n))
    E[:n, :n] = np.eye(n)
    np.testing.assert_allclose(oracle_mod.apply_q(f, E), oracle_mod.form_q(f), atol=1e-15)
    # Q^T C on its top n rows is the unique thin-Q product.
    Q = oracle_mod.form_q(f)
    np.testing.assert_allclose(oracle_mod.apply_qt(f, C)[:n], Q.T @ C, atol=1e-13)


def test_larft_against_explicit_reflectors(oracle_mod):
    """I - Y T Y^T equals the explicit product H_0 H_1 ... H_{n-1}."""
    m, n = 40, 9
    f = oracle_mod.geqr2(inputs.gaussian(m, n, 31))
    Y = oracle_mod.unit_lower(f)
    P = np.eye(m)
    for j in range(n):
        v = Y[:, j]
        P = P @ (np.eye(m) - f.tau[j] * np.outer(v, v))
    T = oracle_mod.larft(f)
    assert np.array_equal(T, np.triu(T))
    np.testing.assert_allclose(np.eye(m) - Y @ T @ Y.T, P, atol=1e-14)


def test_qr_backward_finite_differences(oracle_mod):
    """Adjoint of the sign-normalised thin QR vs central differences (h = 1e-6, FP64)."""
    m, n = 512, 8
    A = inputs.gaussian(m, n, 5000)
    dQ = inputs.gaussian(m, n, 5001)
    dR = np.triu(inputs.gaussian(n, n, 5002))
    Q, R = oracle_mod.qr(A)
    dA = oracle_mod.qr_backward(Q, R, dQ, np.asfortranarray(dR))

    def loss(X):
        q, r = oracle_mod.qr(X)
        return float(np.sum(dQ * q) + np.sum(dR * r))

    h = 1e-6
    for s in range(4):
        E = inputs.gaussian(m, n, 6000 + s)
        fd = (loss(A + h * E) - loss(A - h * E)) / (2 * h)
        an = float(np.sum(dA * E))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


# ------------------------------------------------------------ least squares --
def test_lstsq_straight_line_closed_form(oracle_mod):
    """Fit y = x0 + x1 t through (0, 1), (1, 2), (2, 4): the normal equations
    [[3, 3], [3, 5]] x = [7, 10] give x = (5/6, 3/2), residual (1, -2, 1)/6."""
    A = np.array([[1.0, 0.0], [1.0, 1.0], [1.0, 2.0]])
    b = np.array([1.0, 2.0, 4.0])
    X, rn = oracle_mod.lstsq(A, b)
    np.testing.assert_allclose(X[:, 0], [5.0 / 6.0, 1.5], rtol=0, atol=8 * EPS64)
    assert abs(rn[0] - math.sqrt(6.0) / 6.0) <= 8 * EPS64


def test_lstsq_regression_formula(oracle_mod):
    """Simple linear regression: slope = sum (t - tm)(y - ym) / sum (t - tm)^2, intercept = ym - slope tm."""
    rng = np.random.default_rng(17)
    t = rng.uniform(-3, 3, 50)
    y = 0.7 - 1.3 * t + 0.1 * rng.standard_normal(50)
    A = np.stack([np.ones_like(t), t], axis=1)
    X, rn = oracle_mod.lstsq(A, y)
    tm, ym = t.mean(), y.mean()
    slope = np.sum((t - tm) * (y - ym)) / np.sum((t - tm) ** 2)
    icept = ym - slope * tm
    np.testing.assert_allclose(X[:, 0], [icept, slope], rtol=1e-13)
    assert abs(rn[0] - np.linalg.norm(y - icept - slope * t)) <= 1e-13 * np.linalg.norm(y)


@pytest.mark.parametrize("m,n,k", [(300, 7, 3), (2000, 40, 5), (64, 64, 2)])
def test_lstsq_normal_equations_and_lapack(oracle_mod, m, n, k):
    A = inputs.gaussian(m, n, 500 + n)
    B = inputs.gaussian(m, k, 600 + n)
    X, rn = oracle_mod.lstsq(A, B)
    Rres = A @ X - B
    # The residual is orthogonal to range(A) (the normal equations).
    assert np.abs(A.T @ Rres).max() <= fp64_tol(m, n) * np.linalg.norm(A) * np.linalg.norm(B)
    np.testing.assert_allclose(rn, np.linalg.norm(Rres, axis=0), rtol=fp64_tol(m, n), atol=fp64_tol(m, n))
    Xl = np.linalg.lstsq(A, B, rcond=None)[0]  # LAPACK, run as a library
    kappa = np.linalg.cond(A)
    assert np.abs(X - Xl).max() <= fp64_tol(m, n) * kappa * kappa * np.abs(Xl).max()


def test_lstsq_consistent_system_recovered(oracle_mod):
    m, n = 500, 12
    A = inputs.gaussian(m, n, 701)
    Xt = inputs.gaussian(n, 3, 702)
    X, rn = oracle_mod.lstsq(A, A @ Xt)
    np.testing.assert_allclose(X, Xt, rtol=0, atol=fp64_tol(m, n) * np.linalg.cond(A) * np.abs(Xt).max())
    assert np.all(rn <= fp64_tol(m, n) * np.linalg.norm(A @ Xt, axis=0))

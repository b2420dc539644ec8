"""Parity of the CUDA TSQR path (through the C ABI) with the CPU oracle.

Every input is a seeded synthetic matrix from paper_0808_2664_gb300.inputs;
expected values come only from the oracle.  Tolerances: the FP64 bound
10 * n * eps64 * sqrt(m) on the backward error and orthogonality, and on the
distance to the oracle's R and Q scaled by the condition number; the mixed
form (FP32 storage, FP64 reflectors) uses the same bound with eps32.
"""
import numpy as np
import pytest

from conftest import EPS32, EPS64, assert_colwise_close, fp32_tol, fp64_tol
from paper_0808_2664_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_0808_2664_gb300 as tq  # noqa: E402


def dev(A, dtype=torch.float64):
    return tq.as_colmajor(torch.from_numpy(np.asfortranarray(A)).to("cuda", dtype))


def host(t):
    return t.double().cpu().numpy()


def tol_for(dtype, m, n):
    return fp64_tol(m, n) if dtype == torch.float64 else fp32_tol(m, n)


SHAPES = [
    # (m, n, leaf_rows, arity)
    (4096, 32, 256, 2),   # the small configuration: 16 leaves of 256 rows, binary tree
    (1000, 7, 64, 2),     # ragged: last leaf takes the remainder
    (513, 17, 128, 2),    # remainder < n merges into the previous leaf
    (300, 64, 64, 2),
    (64, 64, 0, 2),       # m = n: one leaf
    (65, 64, 0, 2),
    (5000, 16, 128, 4),   # arity-4 tree with a short last node
    (2049, 1, 256, 2),    # one column
    (777, 3, 32, 3),      # arity 3
    (20000, 64, 256, 8),  # arity 8: 79 leaves, a top node with two children
    (9000, 32, 128, 16),  # arity 16: 70 leaves, a short last node
    (20000, 64, 256, 2),  # several tree levels, odd leaf counts
    (3000, 128, 128, 2),  # the widest n
    (80000, 16, 64, 2),   # 1250 leaves: wide binary levels (two nodes per CTA)
    (4000, 80, 0, 2),     # FP64 n > 64: the 128-column leaf form
]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("m,n,h,q", SHAPES)
def test_factor_and_form_q_match_oracle(oracle_mod, dtype, m, n, h, q):
    A = inputs.gaussian(m, n, seed=1000 + m + n)
    if dtype == torch.float64 and n == 128:
        # FP64 tiles for n = 128 do not fit one CTA's shared memory; such
        # matrices go through caqr_factor with 64-column panels instead.
        with pytest.raises(tq.TsqrError) as ei:
            tq.tsqr_factor(dev(A, dtype), leaf_rows=h, arity=q)
        assert ei.value.code == 5
        return
    Qo, Ro = oracle_mod.qr(A)
    kappa = np.linalg.cond(A)
    Ad = dev(A, dtype)
    R, qt = tq.tsqr_factor(Ad, leaf_rows=h, arity=q)
    Q = qt.form_q()
    assert qt.sync_status() == 0
    Rh, Qh = host(R), host(Q)
    tol = tol_for(dtype, m, n)
    assert np.array_equal(Rh, np.triu(Rh))
    assert np.all(np.diag(Rh) >= 0)
    # Entry by entry, relative to the oracle's column norms (||Qo(:, j)|| = 1).
    assert_colwise_close(Rh, Ro, tol * kappa, "R")
    assert_colwise_close(Qh, Qo, tol * kappa, "Q")
    assert np.linalg.norm(A - Qh @ Rh) / np.linalg.norm(A) <= tol
    assert np.linalg.norm(np.eye(n) - Qh.T @ Qh) <= tol


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("m,n,h,q", [(4096, 32, 256, 2), (1000, 7, 64, 2), (5000, 16, 128, 4), (3000, 128, 128, 2),
                                     (20000, 16, 64, 8)])
def test_apply_qt_and_apply_q(oracle_mod, dtype, m, n, h, q):
    if dtype == torch.float64 and n > 64:
        pytest.skip("FP64 n > 64 is served by caqr_factor")
    A = inputs.gaussian(m, n, seed=7 + m)
    k = 37
    C = inputs.gaussian(m, k, seed=8 + m)
    Qo, Ro = oracle_mod.qr(A)
    Ad = dev(A, dtype)
    R, qt = tq.tsqr_factor(Ad, leaf_rows=h, arity=q)
    tol = tol_for(dtype, m, n)
    # Q^T C: the top n rows are the unique thin-Q product.
    Cd = dev(C, dtype)
    qt.apply_qt(Cd)
    QtC = host(Cd)
    assert np.linalg.norm(QtC[:n] - Qo.T @ C) <= tol * np.linalg.norm(C) * 4
    assert_colwise_close(QtC[:n], Qo.T @ C, 4 * tol, "QtC")
    # Orthogonal: column norms are preserved.
    np.testing.assert_allclose(np.linalg.norm(QtC, axis=0), np.linalg.norm(C, axis=0), rtol=tol * 4)
    # Round trip Q (Q^T C) = C.
    qt.apply_q(Cd)
    assert np.linalg.norm(host(Cd) - C) <= tol * np.linalg.norm(C) * 4
    # Q [X; 0] = Q_thin X.
    X = inputs.gaussian(n, k, seed=9 + m)
    E = np.zeros((m, k))
    E[:n] = X
    Ed = dev(E, dtype)
    qt.apply_q(Ed)
    assert np.linalg.norm(host(Ed) - Qo @ X) <= tol * np.linalg.norm(X) * 4
    assert_colwise_close(host(Ed), Qo @ X, 4 * tol, "QX")
    # Q^T A = [R; 0].
    A2 = dev(A, dtype)
    qt.apply_qt(A2)
    QtA = host(A2)
    assert np.linalg.norm(QtA[:n] - Ro) <= tol * np.linalg.norm(A) * 4
    assert np.linalg.norm(QtA[n:]) <= tol * np.linalg.norm(A) * 4
    assert qt.sync_status() == 0


def test_single_leaf_reflectors_match_oracle(oracle_mod):
    """One leaf is plain Householder QR with the oracle's sign convention: same Y."""
    m, n = 200, 24
    A = inputs.gaussian(m, n, 77)
    f = oracle_mod.geqr2(A)
    Ad = dev(A)
    R, qt = tq.tsqr_factor(Ad, leaf_rows=256)
    assert qt.info()["leaves"] == 1 and qt.info()["levels"] == 0
    Y = host(Ad)
    np.testing.assert_allclose(np.tril(Y, -1), np.tril(f.Y, -1), atol=100 * EPS64)
    np.testing.assert_allclose(np.triu(Y[:n]), np.triu(f.Y[:n]), atol=100 * EPS64 * np.abs(f.Y).max())


def test_tree_shape_and_leaf_height_invariance():
    m, n = 8192, 32
    A = inputs.gaussian(m, n, 4242)
    Rs = []
    for h, q in ((64, 2), (256, 2), (256, 4), (512, 8), (768, 2)):
        R, _ = tq.tsqr_factor(dev(A), leaf_rows=h, arity=q, keep_q=False)
        Rs.append(host(R))
    for R in Rs[1:]:
        assert np.linalg.norm(R - Rs[0]) / np.linalg.norm(Rs[0]) <= fp64_tol(m, n)


def test_row_permutation_invariance():
    m, n = 4096, 16
    A = inputs.gaussian(m, n, 31)
    perm = np.random.default_rng(3).permutation(m)
    R1, _ = tq.tsqr_factor(dev(A), keep_q=False)
    R2, _ = tq.tsqr_factor(dev(A[perm]), keep_q=False)
    assert np.linalg.norm(host(R1) - host(R2)) / np.linalg.norm(host(R1)) <= fp64_tol(m, n)


def test_deterministic_bitwise():
    A = inputs.gaussian(10000, 48, 5)
    outs = []
    for _ in range(2):
        Ad = dev(A)
        R, qt = tq.tsqr_factor(Ad, leaf_rows=256)
        Q = qt.form_q()
        torch.cuda.synchronize()
        outs.append((host(R), host(Q), host(Ad)))
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)


def test_ill_conditioned_backward_stable(oracle_mod):
    """A = G diag(s) W with cond 1e12: backward error and orthogonality stay at the FP64 bound."""
    m, n = 65536, 64
    A = inputs.ill_conditioned(m, n, 2001)
    Ad = dev(A)
    R, qt = tq.tsqr_factor(Ad)
    Q = host(qt.form_q())
    Rh = host(R)
    assert np.linalg.norm(A - Q @ Rh) / np.linalg.norm(A) <= fp64_tol(m, n)
    assert np.linalg.norm(np.eye(n) - Q.T @ Q) <= fp64_tol(m, n)


def test_zero_and_rank_deficient_columns():
    m, n = 1500, 12
    A = inputs.gaussian(m, n, 8)
    A[:, 3] = 0.0
    A[:, 7] = 2.0 * A[:, 1]
    Ad = dev(A)
    R, qt = tq.tsqr_factor(Ad, leaf_rows=128)
    Q, Rh = host(qt.form_q()), host(R)
    assert qt.sync_status() == 0
    assert np.all(np.diag(Rh) >= 0)
    assert np.linalg.norm(A - Q @ Rh) / np.linalg.norm(A) <= fp64_tol(m, n)
    assert np.linalg.norm(np.eye(n) - Q.T @ Q) <= fp64_tol(m, n)


@pytest.mark.parametrize("e", [600, -600])
def test_extreme_scaling(e):
    m, n = 2000, 16
    A = inputs.gaussian(m, n, 12)
    s = 2.0 ** e
    R0, _ = tq.tsqr_factor(dev(A), leaf_rows=256, keep_q=False)
    R1, _ = tq.tsqr_factor(dev(A * s), leaf_rows=256, keep_q=False)
    r0, r1 = host(R0), host(R1) / s
    assert np.all(np.isfinite(r1))
    assert np.linalg.norm(r1 - r0) / np.linalg.norm(r0) <= fp64_tol(m, n)


def test_nonfinite_input_reported():
    A = inputs.gaussian(1024, 8, 1)
    A[500, 2] = np.nan
    R, qt = tq.tsqr_factor(dev(A), leaf_rows=256)
    assert qt.sync_status() == 4  # TSQR_ERR_NONFINITE
    assert qt.sync_status() == 0  # the status word is cleared after reading


def test_argument_errors_and_quick_returns():
    A = dev(inputs.gaussian(10, 20, 1))
    with pytest.raises(tq.TsqrError) as ei:
        tq.tsqr_factor(A)
    assert ei.value.code == -2  # m < n
    L = tq._lib.lib()
    assert L.tsqr_factor(0, 0, None, 1, None, 1, None, None, None) == 0
    assert L.tsqr_factor(5, 3, None, 5, None, 3, None, None, None) == -3
    B = dev(inputs.gaussian(8, 3, 2))
    assert L.tsqr_factor(8, 3, B.data_ptr(), 4, B.data_ptr(), 3, None, None, None) == -4
    assert L.tsqr_apply_qt(None, 1, None, 1, None) == 6  # invalid handle


def test_plan_once_refactor_matches():
    m, n = 12345, 40
    q = tq.tsqr_q_create(m, n, torch.float64, leaf_rows=256)
    for seed in (1, 2):
        A = inputs.gaussian(m, n, seed)
        Ad = dev(A)
        R = q.refactor(Ad)
        R_ref, _ = tq.tsqr_factor(dev(A), leaf_rows=256, keep_q=False)
        assert np.array_equal(host(R), host(R_ref))
        Q = host(q.form_q())
        assert np.linalg.norm(A - Q @ host(R)) / np.linalg.norm(A) <= fp64_tol(m, n)


@pytest.mark.parametrize("mode", ["pinned", "pinned_no_device_q", "pageable"])
@pytest.mark.parametrize("m,n,h", [(100_000, 8, 32), (50_000, 16, 64), (3000, 32, 256)])
def test_factor_form_host_pipeline(oracle_mod, m, n, h, mode):
    """Host-buffer call equals the device calls bitwise and the oracle within the bound; several
    chunks of leaves and a merged last leaf.  Pinned A_host: the leaf kernel loads it itself;
    with no device Q the form stores Q straight into the pinned Q_host; pageable buffers go
    through chunked copies."""
    A = inputs.gaussian(m, n, 21)
    q = tq.tsqr_q_create(m, n, torch.float64, "cuda", leaf_rows=h)
    pin = mode != "pageable"
    Ah = torch.empty((n, m), dtype=torch.float64, pin_memory=pin).t()
    Ah.copy_(torch.from_numpy(A))
    Qh = torch.empty((n, m), dtype=torch.float64, pin_memory=pin).t()
    Rh = torch.empty((n, n), dtype=torch.float64, pin_memory=pin).t()
    Ad, Qd, Rd = tq.colmajor(m, n, torch.float64), tq.colmajor(m, n, torch.float64), tq.colmajor(n, n, torch.float64)
    q.factor_form_host(Ah, Qh, Rh, Ad, None if mode == "pinned_no_device_q" else Qd, Rd)
    torch.cuda.synchronize()
    assert q.sync_status() == 0
    assert torch.equal(Ah, torch.from_numpy(A))  # A_host is only read
    R1, q1 = tq.tsqr_factor(dev(A), leaf_rows=h, arity=q.info()["arity"])
    Q1 = q1.form_q()
    assert torch.equal(Rh, R1.cpu()) and torch.equal(Qh, Q1.cpu()) and torch.equal(Rd, R1)
    if mode != "pinned_no_device_q":
        assert torch.equal(Qd, Q1)
    Qo, Ro = oracle_mod.qr(A)
    tol = fp64_tol(m, n) * np.linalg.cond(A)
    assert np.linalg.norm(Rh.numpy() - Ro) / np.linalg.norm(Ro) <= tol
    assert np.linalg.norm(Qh.numpy() - Qo) <= tol * n ** 0.5
    # The handle keeps the factors: Q^T of a device copy of A gives [R; 0] in its top rows.
    C = dev(A)
    q.apply_qt(C)
    assert torch.equal(C[:n], q1.apply_qt(dev(A))[:n])
    q.destroy()
    q1.destroy()


def test_factor_form_host_fp32_direct():
    """FP32 storage through the host call with pinned buffers and no device Q equals the device
    calls bitwise."""
    m, n, h = 40_000, 32, 256
    A = inputs.gaussian(m, n, 22).astype(np.float32)
    q = tq.tsqr_q_create(m, n, torch.float32, "cuda", leaf_rows=h)
    Ah = torch.empty((n, m), dtype=torch.float32, pin_memory=True).t()
    Ah.copy_(torch.from_numpy(A))
    Qh = torch.empty((n, m), dtype=torch.float32, pin_memory=True).t()
    Rh = torch.empty((n, n), dtype=torch.float32, pin_memory=True).t()
    Ad, Rd = tq.colmajor(m, n, torch.float32), tq.colmajor(n, n, torch.float32)
    q.factor_form_host(Ah, Qh, Rh, Ad, None, Rd)
    torch.cuda.synchronize()
    assert q.sync_status() == 0
    R1, q1 = tq.tsqr_factor(dev(A, torch.float32), leaf_rows=h, arity=q.info()["arity"])
    Q1 = q1.form_q()
    assert torch.equal(Rh, R1.cpu()) and torch.equal(Qh, Q1.cpu())
    q.destroy()
    q1.destroy()


def test_factor_form_host_rejects_pageable_q_without_device_q():
    m, n = 4096, 8
    q = tq.tsqr_q_create(m, n, torch.float64, "cuda")
    Ah = torch.zeros((n, m), dtype=torch.float64, pin_memory=True).t()
    Qh = torch.empty((n, m), dtype=torch.float64).t()  # pageable
    Rh = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
    with pytest.raises(RuntimeError, match="-10"):
        q.factor_form_host(Ah, Qh, Rh, tq.colmajor(m, n, torch.float64), None, tq.colmajor(n, n, torch.float64))
    q.destroy()


def test_leaf_compact_wy_t_matches_oracle(oracle_mod):
    """A single leaf's stored T (tsqr_q_part) equals the oracle's larft of the same
    reflectors, and I - Y T Y^T is the product of the leaf's reflectors."""
    m, n = 300, 24
    A = inputs.gaussian(m, n, 78)
    f = oracle_mod.geqr2(A)
    Ad = dev(A)
    R, qt = tq.tsqr_factor(Ad, leaf_rows=512)
    assert qt.info()["leaves"] == 1
    T = host(qt.part("T", 0, 0))
    tau = host(qt.part("tau", 0, 0))
    To = oracle_mod.larft(f)
    np.testing.assert_allclose(tau, f.tau, rtol=0, atol=64 * EPS64)
    assert_colwise_close(T, To, 256 * n * EPS64, "T")
    assert np.array_equal(T, np.triu(T))
    # I - Y T Y^T against the explicit product of the oracle's reflectors.
    Y = np.tril(host(Ad), -1)[:, :n]
    Y[np.arange(n), np.arange(n)] = 1.0
    H = np.eye(m)
    for j in range(n):
        v = oracle_mod.unit_lower(f)[:, j]
        H = H - f.tau[j] * np.outer(H @ v, v)
    assert np.abs(np.eye(m) - Y @ T @ Y.T - H).max() <= 256 * n * EPS64


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("q", [2, 4])
def test_node_factors_reduce_children(dtype, q):
    """Each tree node's stored Y, T and R (tsqr_q_part): with the structured
    Householder vectors U = [I; Y_1; ...; Y_{q-1}] (Y_b upper triangular),
    (I - U T U^T)^T [R_0; ...; R_{q-1}] = [R_node; 0] and I - U T U^T is orthogonal
    (Eqs. TSQR_binarytree_2/3 with the compact-WY form of the node's reflectors)."""
    m, n, h = 64 * 9 + 5, 16, 64
    A = inputs.gaussian(m, n, 91 + q)
    R, qt = tq.tsqr_factor(dev(A, dtype), leaf_rows=h, arity=q)
    info = qt.info()
    eps = EPS64 if dtype == torch.float64 else EPS32
    items = [info["leaves"]]
    while items[-1] > 1:
        items.append((items[-1] + q - 1) // q)
    for level in range(1, info["levels"] + 1):
        for node in range(items[level]):
            kids = [c for c in range(node * q, min((node + 1) * q, items[level - 1]))]
            stack = np.zeros((q * n, n))
            for b, c in enumerate(kids):
                stack[b * n:(b + 1) * n] = np.triu(host(qt.part("R", level - 1, c)))
            U = np.zeros((q * n, n))
            U[:n] = np.eye(n)
            for b in range(1, q):
                U[b * n:(b + 1) * n] = np.triu(host(qt.part("Y", level, node)[b - 1]))
            T = np.triu(host(qt.part("T", level, node)))
            Hn = np.eye(q * n) - U @ T @ U.T
            Rn = np.triu(host(qt.part("R", level, node)))
            out = Hn.T @ stack
            scale = np.linalg.norm(stack)
            assert np.abs(out[:n] - Rn).max() <= 64 * n * eps * scale, (level, node)
            assert np.abs(out[n:]).max() <= 64 * n * eps * scale, (level, node)
            assert np.abs(Hn.T @ Hn - np.eye(q * n)).max() <= 64 * n * eps, (level, node)
    qt.destroy()


def _decimal_reflector(alpha, ssq):
    """beta, tau, scale of x = [alpha; t] with ||t||^2 = ssq, in 60-digit decimal arithmetic."""
    from decimal import Decimal, getcontext

    getcontext().prec = 60
    a, s = Decimal(float(alpha)), Decimal(float(ssq))
    nrm = (a * a + s).sqrt()
    beta = -nrm if a >= 0 else nrm
    d = a - beta
    return beta, (beta - a) / beta, 1 / d


@pytest.mark.parametrize("fast", [0, 1])
def test_reflector_generation_accuracy(fast):
    """The reflector of the leaf and node kernels (both the IEEE form and the short-latency
    form of each column's serial step) against 60-digit decimal arithmetic: beta, tau and
    scale within a few FP64 ulps, and tau u^T u = tau (1 + scale^2 ssq) = 2 (H orthogonal)."""
    from decimal import Decimal

    rng = np.random.default_rng(2024 + fast)
    cnt = 6000
    alpha = rng.choice([-1.0, 1.0], cnt) * 10.0 ** rng.uniform(-14, 14, cnt)
    ssq = 10.0 ** rng.uniform(-28, 28, cnt)
    # Some inputs outside the fast form's safe range (it falls back to the IEEE form there).
    alpha[:200] *= 1e20
    ssq[200:400] *= 1e-40
    ad = torch.from_numpy(alpha).cuda()
    sd = torch.from_numpy(ssq).cuda()
    out = torch.empty(3 * cnt, dtype=torch.float64, device="cuda")
    L = tq._lib.lib()
    import ctypes

    rc = L.tsqr_test_reflectors(cnt, ctypes.c_void_p(ad.data_ptr()), ctypes.c_void_p(sd.data_ptr()), fast,
                                ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    got = out.cpu().numpy().reshape(cnt, 3)
    ulps = 16 if fast else 8
    worst = 0.0
    for i in range(cnt):
        ex = _decimal_reflector(alpha[i], ssq[i])
        for k in range(3):
            e = float(ex[k])
            err = abs(got[i, k] - e) / np.spacing(abs(e))
            worst = max(worst, err)
            assert err <= ulps, (i, k, alpha[i], ssq[i], got[i, k], e, err)
        tau, scale = Decimal(float(got[i, 1])), Decimal(float(got[i, 2]))
        ident = abs(tau * (1 + scale * scale * Decimal(float(ssq[i]))) - 2)
        assert ident <= Decimal(16 * 2.0 ** -52), (i, float(ident))


REC_SHAPES = [(4096, 32, 256, 2), (1000, 7, 64, 2), (20000, 64, 0, 4), (300, 64, 0, 2), (2049, 1, 256, 2),
              (777, 3, 32, 3), (513, 17, 128, 2), (65, 64, 0, 2), (9000, 33, 128, 4)]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("m,n,h,q", REC_SHAPES)
def test_recursive_leaf_matches_oracle(oracle_mod, dtype, m, n, h, q):
    """Leaves factored by the recursive (RGEQR3) leaf QR: same R, Q and Q^T C as the oracle."""
    A = inputs.gaussian(m, n, seed=5100 + m + n)
    if dtype == torch.float32:
        A = A.astype(np.float32).astype(np.float64)
    Qo, Ro = oracle_mod.qr(A)
    kappa = np.linalg.cond(Ro)
    tol = tol_for(dtype, m, n)
    Ad = dev(A, dtype)
    R, qt = tq.tsqr_factor(Ad, leaf_rows=h, arity=q, flags=tq.FLAG_RECURSIVE_LEAF)
    Q = qt.form_q()
    assert qt.sync_status() == 0
    Rh, Qh = host(R), host(Q)
    assert np.all(np.diag(Rh) >= 0)
    assert_colwise_close(Rh, Ro, tol * kappa, "R")
    assert_colwise_close(Qh, Qo, tol * kappa, "Q")
    C = inputs.gaussian(m, 9, seed=5200 + n)
    Cd = dev(C, dtype)
    qt.apply_qt(Cd)
    assert_colwise_close(host(Cd)[:n], Qo.T @ C, 4 * tol * kappa, "QtC")
    qt.destroy()


def test_recursive_leaf_t_matches_oracle(oracle_mod):
    """One recursive leaf: its merged T equals the oracle's larft of the same reflectors."""
    m, n = 300, 40
    A = inputs.gaussian(m, n, 5300)
    f = oracle_mod.geqr2(A)
    Ad = dev(A)
    R, qt = tq.tsqr_factor(Ad, leaf_rows=512, flags=tq.FLAG_RECURSIVE_LEAF)
    assert qt.info()["leaves"] == 1
    np.testing.assert_allclose(np.tril(host(Ad), -1), np.tril(f.Y, -1), atol=100 * EPS64)
    T = host(qt.part("T", 0, 0))
    assert_colwise_close(T, oracle_mod.larft(f), 256 * n * EPS64, "T")
    np.testing.assert_allclose(host(qt.part("tau", 0, 0)), f.tau, rtol=0, atol=64 * EPS64)
    qt.destroy()


def test_recursive_leaf_rejects_hybrid_and_wide():
    with pytest.raises(tq.TsqrError) as ei:
        tq.tsqr_q_create(4096, 16, torch.float64, flags=tq.FLAG_RECURSIVE_LEAF | tq.FLAG_HYBRID_TREE)
    assert ei.value.code == 5
    with pytest.raises(tq.TsqrError) as ei:
        tq.tsqr_q_create(4096, 100, torch.float32, flags=tq.FLAG_RECURSIVE_LEAF)
    assert ei.value.code == 5

"""The hybrid and flat reduction trees (Section 2.1) through the C ABI, against the CPU oracle.

Flat tree: one CTA streams every leaf, each later leaf factored stacked under
the running R (sequential TSQR).  Hybrid: one such chain per resident CTA, a
q-ary tree over the chains.  By uniqueness of the sign-normalised QR
(Section 2.1, after Eq. TSQR_binarytree_4) R and the thin Q equal the
oracle's whatever the tree; Q^T C is unique in its top n rows.  Tolerance:
10 n eps sqrt(m) (eps of the storage type) times cond(A), entry by entry
relative to the oracle's column norms.
"""
import numpy as np
import pytest

from conftest import assert_colwise_close, fp32_tol, fp64_tol
from paper_0808_2664_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_0808_2664_gb300 as tq  # noqa: E402


def dev(A, dtype=torch.float64):
    return tq.as_colmajor(torch.from_numpy(np.asfortranarray(A)).to("cuda", dtype))


def host(t):
    return t.double().cpu().numpy()


CASES = [
    # (m, n, leaf_rows, arity, flags)
    (1_000_000, 16, 64, 4, "hybrid"),   # chains of several leaves, four-triangle tree over chains
    (300_000, 64, 0, 2, "hybrid"),      # default leaf height (n rows below the plain default)
    (20000, 32, 256, 4, "flat"),        # one chain: sequential TSQR
    (5000, 7, 64, 2, "flat"),           # ragged: merged last leaf in a stacked step
    (777, 1, 32, 2, "flat"),            # one column
    (64, 64, 0, 2, "hybrid"),           # a single leaf
    (100_000, 128, 0, 2, "hybrid"),     # the widest n
]


def _flags(kind):
    return tq.FLAG_FLAT_TREE if kind == "flat" else tq.FLAG_HYBRID_TREE


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("m,n,h,q,kind", CASES)
def test_hybrid_factor_form_apply_match_oracle(oracle_mod, dtype, m, n, h, q, kind):
    if dtype == torch.float64 and n > 64:
        pytest.skip("FP64 n > 64 tiles do not fit with the stacked rows")
    A = inputs.gaussian(m, n, seed=3100 + m % 1000 + n)
    if dtype == torch.float32:
        A = A.astype(np.float32).astype(np.float64)
    Qo, Ro = oracle_mod.qr(A)
    kappa = np.linalg.cond(Ro)
    tol = (fp64_tol if dtype == torch.float64 else fp32_tol)(m, n)
    qt = tq.tsqr_q_create(m, n, dtype, leaf_rows=h, arity=q, flags=_flags(kind))
    ch = qt.chains()
    info = qt.info()
    if kind == "flat":
        assert ch["chains"] == 1 and ch["leaves_per_chain"] == info["leaves"]
    Ad = dev(A, dtype)
    R = qt.refactor(Ad)
    Q = qt.form_q()
    assert qt.sync_status() == 0
    Rh, Qh = host(R), host(Q)
    assert np.all(np.diag(Rh) >= 0) and np.array_equal(Rh, np.triu(Rh))
    assert_colwise_close(Rh, Ro, tol * kappa, "R")
    assert_colwise_close(Qh, Qo, tol * kappa, "Q")
    # Q^T C: unique top n rows, column norms kept; Q (Q^T C) = C.
    k = 37
    C = inputs.gaussian(m, k, seed=3200 + n)
    if dtype == torch.float32:
        C = C.astype(np.float32).astype(np.float64)
    Cd = dev(C, dtype)
    qt.apply_qt(Cd)
    QtC = host(Cd)
    assert_colwise_close(QtC[:n], Qo.T @ C, 4 * tol * kappa, "QtC")
    np.testing.assert_allclose(np.linalg.norm(QtC, axis=0), np.linalg.norm(C, axis=0), rtol=4 * tol)
    qt.apply_q(Cd)
    assert_colwise_close(host(Cd), C, 4 * tol, "QQtC")
    # Q^T A = [R; 0].
    A2 = dev(A, dtype)
    qt.apply_qt(A2)
    QtA = host(A2)
    assert_colwise_close(QtA[:n], Rh, 4 * tol, "QtA")
    if m > n:
        assert np.abs(QtA[n:]).max() <= 4 * tol * np.linalg.norm(A, axis=0).max()
    qt.destroy()


def test_hybrid_chains_span_the_gpu():
    m, n = 4_194_304, 64
    qt = tq.tsqr_q_create(m, n, torch.float64, flags=tq.FLAG_HYBRID_TREE)
    ch, info = qt.chains(), qt.info()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert ch["leaves_per_chain"] > 1
    assert sms // 2 <= ch["chains"] <= 4 * sms
    assert info["levels"] <= 5
    qt.destroy()


def test_hybrid_same_r_as_qary_and_deterministic():
    m, n = 200_000, 48
    A = inputs.gaussian(m, n, 3300)
    R1, _ = tq.tsqr_factor(dev(A), keep_q=False)
    outs = []
    for _ in range(2):
        Ad = dev(A)
        R2, q2 = tq.tsqr_factor(Ad, flags=tq.FLAG_HYBRID_TREE)
        outs.append((host(R2), host(q2.form_q())))
        q2.destroy()
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert_colwise_close(outs[0][0], host(R1), fp64_tol(m, n), "R")


def test_hybrid_unsupported_combinations():
    with pytest.raises(tq.TsqrError) as ei:
        tq.tsqr_q_create(4096, 32, torch.float32, flags=tq.FLAG_HYBRID_TREE | tq.FLAG_APPLY_BF16X3)
    assert ei.value.code == 5
    q = tq.tsqr_q_create(4096, 8, torch.float64, flags=tq.FLAG_HYBRID_TREE)
    Ah = torch.zeros((8, 4096), dtype=torch.float64).t()
    Qh = torch.zeros((8, 4096), dtype=torch.float64).t()
    Rh = torch.zeros((8, 8), dtype=torch.float64).t()
    with pytest.raises(tq.TsqrError) as ei:
        q.factor_form_host(Ah, Qh, Rh, tq.colmajor(4096, 8), tq.colmajor(4096, 8), tq.colmajor(8, 8))
    assert ei.value.code == 5
    q.destroy()

"""Parity of the CUDA CAQR path (TSQR panels + trailing updates) with the CPU oracle.

CAQR returns the same factorisation as unblocked Householder QR once diag(R)
is made non-negative, so R and the thin Q are compared with the oracle's, and
Q^T C's top n rows with the oracle's thin-Q product.  Tolerance: the FP64
bound 10 * n * eps * sqrt(m), times the condition number for R and Q.
"""
import numpy as np
import pytest

from conftest import fp64_tol
from paper_0808_2664_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_0808_2664_gb300 as tq  # noqa: E402


def dev(A):
    return tq.as_colmajor(torch.from_numpy(np.asfortranarray(A)).to("cuda"))


def host(t):
    return t.double().cpu().numpy()


@pytest.mark.parametrize("m,n,b,h", [
    (256, 256, 32, 0),     # square, several panels
    (512, 512, 64, 128),   # square, panel width 64
    (1000, 200, 48, 0),    # tall, ragged last panel
    (3000, 128, 64, 0),    # tall n = 128 in FP64 via two 64-column panels
    (300, 300, 7, 64),     # odd panel width
    (120, 120, 120, 0),    # one panel: CAQR reduces to TSQR
    (1300, 1200, 64, 0),   # wide trailing updates: two column halves on two streams
])
def test_caqr_matches_oracle(oracle_mod, m, n, b, h):
    A = inputs.uniform(m, n, seed=3000 + m + n)
    Qo, Ro = oracle_mod.qr(A)
    kappa = np.linalg.cond(A)
    Ad = dev(A)
    q = tq.caqr_factor(Ad, b=b, leaf_rows=h)
    Q = q.form_q()
    assert q.sync_status() == 0
    R = np.triu(host(Ad)[:n, :n])
    Qh = host(Q)
    tol = fp64_tol(m, n)
    assert np.all(np.diag(R) >= 0)
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= tol * kappa
    assert np.linalg.norm(Qh - Qo) <= tol * kappa * np.sqrt(n)
    assert np.linalg.norm(A - Qh @ R) / np.linalg.norm(A) <= tol
    assert np.linalg.norm(np.eye(n) - Qh.T @ Qh) <= tol
    # Q^T C: top n rows are unique; Q (Q^T C) = C.
    C = inputs.gaussian(m, 19, seed=5)
    Cd = dev(C)
    q.apply_qt(Cd)
    assert np.linalg.norm(host(Cd)[:n] - Qo.T @ C) <= 4 * tol * kappa * np.linalg.norm(C)
    q.apply_q(Cd)
    assert np.linalg.norm(host(Cd) - C) <= 4 * tol * np.linalg.norm(C)


def test_caqr_ill_conditioned_backward_stable():
    m = n = 384
    A = inputs.ill_conditioned(m, n, 31, cond=1e12)
    Ad = dev(A)
    q = tq.caqr_factor(Ad, b=64)
    Q = host(q.form_q())
    R = np.triu(host(Ad)[:n, :n])
    assert np.linalg.norm(A - Q @ R) / np.linalg.norm(A) <= fp64_tol(m, n)
    assert np.linalg.norm(np.eye(n) - Q.T @ Q) <= fp64_tol(m, n)


def test_caqr_argument_errors():
    A = dev(inputs.uniform(64, 64, 1))
    with pytest.raises(tq.TsqrError) as ei:
        tq.caqr_factor(A, b=0)
    assert ei.value.code == -5
    with pytest.raises(tq.TsqrError) as ei:
        tq.caqr_factor(A, b=16, update_precision=7)
    assert ei.value.code == -6


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3"])
def test_refactor_graph_replay_matches_direct(prec):
    """caqr_refactor's captured panel loop gives bitwise the direct loop's result,
    on replay, on a second buffer (a new capture) and with stage timing on (direct)."""
    m, n, b = 1500, 1280, 64  # the first FP64 trailing updates are wide enough to split
    A = inputs.uniform(m, n, seed=3500)
    dt = torch.float64 if prec == "fp64" else torch.float32
    upd = {"fp64": tq.PREC_FP64, "fp32": tq.PREC_FP32, "bf16x3": tq.UPDATE_BF16X3}[prec]

    def fresh():
        return tq.as_colmajor(torch.from_numpy(np.asfortranarray(A)).to("cuda", dt))

    A0 = fresh()
    tq.caqr_factor(A0, b=b, update_precision=upd, keep_q=False)
    ref = A0.cpu()
    q = tq.caqr_q_create(m, n, b, dt, "cuda", update_precision=upd)
    A1, A2 = fresh(), fresh()
    src = A1.clone()
    for rep in range(2):  # capture, then replay on restored contents
        A1.copy_(src)
        q.refactor(A1)
        torch.cuda.synchronize()
        assert torch.equal(A1.cpu(), ref), rep
    q.refactor(A2)  # another buffer: captured anew
    assert torch.equal(A2.cpu(), ref)
    q.set_timing(True)
    A1.copy_(src)
    q.refactor(A1)
    q.stage_times()
    q.set_timing(False)
    assert torch.equal(A1.cpu(), ref)
    assert q.sync_status() == 0
    Q = q.form_q().double().cpu().numpy()
    R = np.triu(A2.double().cpu().numpy()[:n, :n])
    assert np.linalg.norm(A - Q @ R) / np.linalg.norm(A) <= 1e-3

"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

  * 4,194,304 x 64 FP64, iid N(0, 1), default plan (leaf height and arity of
    the planner): R and the thin Q against the CPU oracle entry by entry,
    relative to the oracle's column norms, within 10 n eps sqrt(m) cond(A);
  * the same shape, ill-conditioned A = G diag(s) W (cond 1e12): backward
    error and orthogonality within 10 n eps sqrt(m) (R itself is not unique
    to that accuracy);
  * CAQR FP64 on a square 4096 x 4096 U[-1, 1] matrix with 64-column panels:
    R against the oracle entry by entry, and the backward error.
Uniqueness of the sign-normalised QR factorisation (Section 2.1, after
Eq. TSQR_binarytree_4) is what makes the entry-by-entry comparison valid for
any tree.  These tests take tens of seconds each (the oracle runs on the
host's cores).
"""
import numpy as np
import pytest

from conftest import assert_colwise_close, fp64_tol
from paper_0808_2664_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_0808_2664_gb300 as tq  # noqa: E402

M_FULL, N_FULL = 4_194_304, 64


def _device_errors(A_dev, Q, R):
    """Backward error and orthogonality in FP64 on the device."""
    berr = (torch.linalg.norm(A_dev - Q @ R) / torch.linalg.norm(A_dev)).item()
    n = Q.shape[1]
    orth = torch.linalg.norm(torch.eye(n, dtype=Q.dtype, device=Q.device) - Q.t() @ Q).item()
    return berr, orth


def test_full_size_gaussian_matches_oracle(oracle_mod):
    m, n = M_FULL, N_FULL
    A = inputs.gaussian(m, n, seed=2001)
    A0 = tq.as_colmajor(torch.from_numpy(A).cuda())
    Ad = A0.clone(memory_format=torch.preserve_format)
    Ad = tq.as_colmajor(Ad)
    R, q = tq.tsqr_factor(Ad)
    info = q.info()
    assert info["leaves"] > 10000 and info["levels"] >= 6
    Q = q.form_q()
    assert q.sync_status() == 0
    tol = fp64_tol(m, n)
    berr, orth = _device_errors(A0, Q, R)
    assert berr <= tol and orth <= tol, (berr, orth, tol)
    Rh = R.cpu().numpy()
    Qh = Q.cpu().numpy()
    del A0, Ad, Q
    torch.cuda.empty_cache()
    Qo, Ro = oracle_mod.qr(A)
    kappa = np.linalg.cond(Ro)
    assert_colwise_close(Rh, Ro, tol * kappa, "R")
    assert_colwise_close(Qh, Qo, tol * kappa, "Q")
    q.destroy()


def test_full_size_ill_conditioned_backward_stable():
    m, n = M_FULL, N_FULL
    A = inputs.ill_conditioned(m, n, seed=2002)
    A0 = tq.as_colmajor(torch.from_numpy(A).cuda())
    del A
    Ad = tq.as_colmajor(A0.clone(memory_format=torch.preserve_format))
    R, q = tq.tsqr_factor(Ad)
    Q = q.form_q()
    assert q.sync_status() == 0
    assert torch.all(torch.diagonal(R) >= 0)
    berr, orth = _device_errors(A0, Q, R)
    tol = fp64_tol(m, n)
    assert berr <= tol and orth <= tol, (berr, orth, tol)
    q.destroy()


def test_caqr_fp64_4096_matches_oracle(oracle_mod):
    n, b = 4096, 64
    A = inputs.uniform(n, n, seed=3004)
    Ad = tq.as_colmajor(torch.from_numpy(A).cuda())
    q = tq.caqr_factor(Ad, b=b)
    Q = q.form_q()
    assert q.sync_status() == 0
    R = torch.triu(Ad)
    A0 = torch.from_numpy(A).cuda()
    berr, orth = _device_errors(A0, Q, R)
    tol = fp64_tol(n, n)
    assert berr <= tol and orth <= tol, (berr, orth, tol)
    Rh = R.cpu().numpy()
    _, Ro = oracle_mod.qr(A, want_q=False)
    kappa = np.linalg.cond(Ro)
    assert_colwise_close(Rh, Ro, tol * kappa, "R")
    # The Gram matrix needs no condition number: ||R^T R - A^T A|| <= (2 berr + orth) ||A||^2.
    gram = np.linalg.norm(Rh.T @ Rh - Ro.T @ Ro) / np.linalg.norm(Ro) ** 2
    assert gram <= 3 * tol, gram
    q.destroy()

"""CAQR with FP32 storage: FP32 trailing updates and 3xBF16 tensor-core (tcgen05) trailing updates.

Reflector generation stays in FP64 in both forms.  Tolerances are derived
from the product arithmetic: FP32 products, eps32 = 2^-23; three BF16
products (hi*hi + hi*lo + lo*hi), relative product error about 2^-16.  The
backward error and orthogonality are checked against
10 * n * eps * sqrt(m); R against the FP64 oracle within that bound times
the condition number.
"""
import numpy as np
import pytest

from conftest import fp32_tol
from paper_0808_2664_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_0808_2664_gb300 as tq  # noqa: E402

EPS_BF16X3 = 2.0 ** -16


def bf16x3_tol(m, n):
    return 10.0 * n * EPS_BF16X3 * m ** 0.5


def dev32(A):
    return tq.as_colmajor(torch.from_numpy(np.asfortranarray(A)).to("cuda", torch.float32))


@pytest.mark.parametrize("upd", ["fp32", "bf16x3"])
@pytest.mark.parametrize("m,n,b", [(256, 256, 64), (1000, 300, 64), (777, 200, 48), (2048, 128, 32)])
def test_caqr_fp32_storage_matches_oracle(oracle_mod, upd, m, n, b):
    A = inputs.uniform(m, n, seed=9000 + m + n)
    Qo, Ro = oracle_mod.qr(A)
    kappa = np.linalg.cond(A)
    Ad = dev32(A)
    prec = tq.PREC_FP32 if upd == "fp32" else tq.UPDATE_BF16X3
    q = tq.caqr_factor(Ad, b=b, update_precision=prec)
    Q = q.form_q().double().cpu().numpy()
    assert q.sync_status() == 0
    R = np.triu(Ad.double().cpu().numpy()[:n, :n])
    tol = fp32_tol(m, n) if upd == "fp32" else bf16x3_tol(m, n)
    assert np.all(np.diag(R) >= 0)
    assert np.linalg.norm(A - Q @ R) / np.linalg.norm(A) <= tol
    assert np.linalg.norm(np.eye(n) - Q.T @ Q) <= max(tol, fp32_tol(m, n))
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= tol * kappa


def test_bf16x3_update_close_to_fp32_update():
    """The tensor-core trailing update agrees with the FP32 CUDA-core one to the BF16x3 bound."""
    m = n = 512
    A = inputs.uniform(m, n, 9100)
    A1, A2 = dev32(A), dev32(A)
    tq.caqr_factor(A1, b=64, update_precision=tq.PREC_FP32, keep_q=False)
    tq.caqr_factor(A2, b=64, update_precision=tq.UPDATE_BF16X3, keep_q=False)
    r1 = np.triu(A1.double().cpu().numpy())
    r2 = np.triu(A2.double().cpu().numpy())
    assert np.linalg.norm(r1 - r2) / np.linalg.norm(r1) <= bf16x3_tol(m, n) * np.linalg.cond(A)

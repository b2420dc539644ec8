"""CAQR and single trailing updates with FP32 storage: FP32 products and 3xBF16 or
3xTF32 tensor-core (tcgen05) products, reflector generation in FP64 in every form.

Bounds (derived from the product arithmetic, not from measurements):
  * one trailing update C <- (I - Y T^T Y^T) C (Section 3.1) is compared with
    the oracle's FP64 Q^T C entry by entry:
        |dC_ij| <= 2 eps (|Y| |T|^T |Y|^T |C|)_ij,
    eps = 2^-16 for three BF16 products, 2^-18 for three TF32 products (whose
    error floor is the tensor cores' FP32 accumulation), 2^-23 for FP32
    products, with the
    oracle's Y and T.  A 3xBF16 product loses at most about 3 * 2^-16 of
    |x y|; a kernel that dropped its hi*lo or lo*hi term would lose about
    2^-9 of it, which puts such errors at 20 to 50 times this bound (an
    emulation of both on these shapes gives 0.1-0.2 and 24-55 times 2^-16 of
    the right-hand side); with several leaves only the top n rows are unique
    and the column-wise form |dC_ij| <= 2 eps ||C(:, j)||_2 is used;
  * whole CAQR: backward error <= c sqrt(n) eps (conftest.caqr_mixed_tol:
    c = 2 for FP32, c = 1 for 3xBF16), orthogonality of the formed Q <= n eps32
    (Q comes from the FP32-stored reflectors, whatever the update arithmetic),
    and R against the oracle through its Gram matrix,
        ||R^T R - Ro^T Ro||_F / ||Ro||_F^2 <= 2 (backward bound) + orthogonality bound,
    which holds for any A = QR with that backward error and needs no cond(A).
"""
import numpy as np
import pytest

from conftest import EPS32, EPS_BF16X3, EPS_TF32X3, assert_colwise_close, caqr_mixed_tol
from paper_0808_2664_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_0808_2664_gb300 as tq  # noqa: E402

C_FP32, C_BF16X3 = 2.0, 1.0


def dev32(A):
    return tq.as_colmajor(torch.from_numpy(np.asfortranarray(A)).to("cuda", torch.float32))


def f32_exact(X):
    """X rounded to FP32 and back: the matrix the FP32 path and the oracle both see."""
    return np.asarray(X, dtype=np.float32).astype(np.float64)


def bounds(upd, n):
    if upd == "fp32":
        return caqr_mixed_tol(n, EPS32, C_FP32)
    if upd == "tf32x3":
        return caqr_mixed_tol(n, EPS_TF32X3, C_BF16X3)
    return caqr_mixed_tol(n, EPS_BF16X3, C_BF16X3)


PREC = {"fp32": tq.PREC_FP32, "bf16x3": tq.UPDATE_BF16X3, "tf32x3": tq.UPDATE_TF32X3}
FLAGS = {"fp32": 0, "bf16x3": tq.FLAG_APPLY_BF16X3, "tf32x3": tq.FLAG_APPLY_TF32X3}
EPS = {"fp32": EPS32, "bf16x3": EPS_BF16X3, "tf32x3": EPS_TF32X3}


@pytest.mark.parametrize("upd", ["fp32", "bf16x3", "tf32x3"])
@pytest.mark.parametrize("m,n,b", [(256, 256, 64), (1000, 300, 64), (777, 200, 48), (2048, 128, 32), (1536, 1024, 64)])
def test_caqr_fp32_storage_matches_oracle(oracle_mod, upd, m, n, b):
    A = f32_exact(inputs.uniform(m, n, seed=9000 + m + n))
    Qo, Ro = oracle_mod.qr(A)
    Ad = dev32(A)
    q = tq.caqr_factor(Ad, b=b, update_precision=PREC[upd])
    Q = q.form_q().double().cpu().numpy()
    assert q.sync_status() == 0
    R = np.triu(Ad.double().cpu().numpy()[:n, :n])
    tol = bounds(upd, n)
    orth_tol = n * EPS32
    assert np.all(np.diag(R) >= 0)
    berr = np.linalg.norm(A - Q @ R) / np.linalg.norm(A)
    assert berr <= tol, (berr, tol)
    orth = np.linalg.norm(np.eye(n) - Q.T @ Q)
    assert orth <= orth_tol, (orth, orth_tol)
    gram = np.linalg.norm(R.T @ R - Ro.T @ Ro) / np.linalg.norm(Ro) ** 2
    assert gram <= 2 * tol + orth_tol, (gram, 2 * tol + orth_tol)


def test_bf16x3_update_close_to_fp32_update():
    """The tensor-core trailing update and the FP32 CUDA-core one give Gram matrices within the 3xBF16 bound."""
    m = n = 512
    A = f32_exact(inputs.uniform(m, n, 9100))
    A1, A2 = dev32(A), dev32(A)
    tq.caqr_factor(A1, b=64, update_precision=tq.PREC_FP32, keep_q=False)
    tq.caqr_factor(A2, b=64, update_precision=tq.UPDATE_BF16X3, keep_q=False)
    r1 = np.triu(A1.double().cpu().numpy())
    r2 = np.triu(A2.double().cpu().numpy())
    gram = np.linalg.norm(r1.T @ r1 - r2.T @ r2) / np.linalg.norm(r1) ** 2
    assert gram <= 2 * (bounds("bf16x3", n) + bounds("fp32", n)), gram


def _single_update(oracle_mod, m, n, k, h, upd, seed):
    A = f32_exact(inputs.gaussian(m, n, seed))
    C = f32_exact(inputs.gaussian(m, k, seed + 1))
    q = tq.tsqr_q_create(m, n, torch.float32, leaf_rows=h, arity=2, flags=FLAGS[upd])
    q.refactor(dev32(A))
    Cd = dev32(C)
    q.apply_qt(Cd)
    got = Cd.double().cpu().numpy()
    assert q.sync_status() == 0
    f = oracle_mod.geqr2(A)
    want = oracle_mod.apply_qt(f, C)
    return A, C, q, f, got, want


@pytest.mark.parametrize("upd", ["bf16x3", "tf32x3", "fp32"])
@pytest.mark.parametrize("m,k", [(512, 256), (450, 200), (130, 64), (512, 1000)])
def test_single_leaf_update_elementwise(oracle_mod, upd, m, k):
    """One leaf (the panel is one row block): its reflectors are the oracle's, so every
    row of Q^T C is unique and is compared entry by entry with the FP64 oracle."""
    n = 64
    A, C, q, f, got, want = _single_update(oracle_mod, m, n, k, m, upd, 7100 + m + k)
    assert q.info()["leaves"] == 1
    Y = oracle_mod.unit_lower(f)
    T = oracle_mod.larft(f)
    rhs = np.abs(Y) @ (np.abs(T).T @ (np.abs(Y).T @ np.abs(C)))
    eps = EPS[upd]
    # The product's own error (2 eps), one FP32 rounding of each of the three
    # stored factors Y, T, Y^T (3 u32, u32 = EPS32 / 2), and one rounding of
    # each stored result entry.
    bound = (2 * eps + 1.5 * EPS32) * rhs + EPS32 * np.abs(want)
    ratio = np.abs(got - want) / bound
    i, j = np.unravel_index(np.argmax(ratio), ratio.shape)
    assert ratio[i, j] <= 1.0, (i, j, got[i, j], want[i, j], bound[i, j])
    q.destroy()


@pytest.mark.parametrize("upd", ["bf16x3", "tf32x3", "fp32"])
@pytest.mark.parametrize("m,n,k,h", [(4096, 64, 300, 512), (3000, 32, 129, 256), (20000, 64, 128, 512)])
def test_multi_leaf_update_columnwise(oracle_mod, upd, m, n, k, h):
    """Several leaves and a binary tree: the top n rows of Q^T C (the unique part)
    against the oracle, column-wise; the rest keeps each column's norm."""
    A, C, q, f, got, want = _single_update(oracle_mod, m, n, k, h, upd, 7300 + m + k)
    assert q.info()["leaves"] > 1
    eps = EPS[upd]
    tol = 2 * eps + 4 * n * EPS32  # the update, plus the FP32 tree levels
    assert_colwise_close(got[:n], want[:n], tol, "QtC")
    np.testing.assert_allclose(np.linalg.norm(got, axis=0), np.linalg.norm(C, axis=0), rtol=tol)
    q.destroy()


def test_bf16x3_flag_rejected_where_unsupported():
    with pytest.raises(tq.TsqrError) as ei:
        tq.tsqr_q_create(1000, 16, torch.float64, flags=tq.FLAG_APPLY_BF16X3)
    assert ei.value.code == 5
    with pytest.raises(tq.TsqrError) as ei:
        tq.tsqr_q_create(1000, 100, torch.float32, flags=tq.FLAG_APPLY_BF16X3)
    assert ei.value.code == 5
    with pytest.raises(tq.TsqrError) as ei:
        tq.tsqr_q_create(1000, 16, torch.float32, flags=1 << 10)
    assert ei.value.code == -4


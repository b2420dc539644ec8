"""Batched uneven TSQR (one persistent launch, graph replay, autotuner) against the oracle."""
import numpy as np
import pytest

from conftest import fp32_tol, fp64_tol
from paper_0808_2664_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_0808_2664_gb300 as tq  # noqa: E402


def dev(A, dtype):
    return tq.as_colmajor(torch.from_numpy(np.asfortranarray(A)).to("cuda", dtype))


def shapes(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.choice([1, 3, 16, 32, 64]))
        m = int(rng.integers(max(n, 64), 6000))
        out.append((m, n))
    return out


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("arity,tile_kb", [(2, 0), (4, 32), (3, 0)])
def test_batch_matches_oracle(oracle_mod, dtype, arity, tile_kb):
    sh = shapes(24, 7 + arity)
    mats = [inputs.gaussian(m, n, 100 + i) for i, (m, n) in enumerate(sh)]
    As = [dev(A, dtype) for A in mats]
    b = tq.Batch(As, arity=arity, tile_kb=tile_kb)
    for rep in range(2):  # graph replay twice; the second run refactors restored inputs
        if rep:
            for A_d, A in zip(As, mats):
                A_d.copy_(dev(A, dtype))
        b.factor(graph=True)
        assert b.sync_status() == 0
        for (m, n), A, R in zip(sh, mats, b.R):
            _, Ro = oracle_mod.qr(A, want_q=False)
            tol = fp64_tol(m, n) if dtype == torch.float64 else fp32_tol(m, n)
            Rh = R.double().cpu().numpy()
            assert np.all(np.diag(Rh) >= 0)
            assert np.linalg.norm(Rh - Ro) / np.linalg.norm(Ro) <= tol * np.linalg.cond(A)


def test_batch_matches_plain_path_and_autotune():
    sh = inputs.batched_shapes(64, 4, m_lo=1024, m_hi=8192)
    mats = [inputs.gaussian(m, n, 900 + i) for i, (m, n) in enumerate(sh)]
    As = [dev(A, torch.float32) for A in mats]
    b = tq.Batch(As, autotune=True)
    info = b.info()
    assert info["arity"] in (2, 4, 8) and info["tile_kb"] > 0
    for A_d, A in zip(As, mats):
        A_d.copy_(dev(A, torch.float32))
    b.factor(graph=False)
    assert b.sync_status() == 0
    for (m, n), A, R in zip(sh, mats, b.R):
        R_ref, _ = tq.tsqr_factor(dev(A, torch.float32), keep_q=False)
        r, rr = R.double().cpu().numpy(), R_ref.double().cpu().numpy()
        assert np.linalg.norm(r - rr) / np.linalg.norm(rr) <= 4 * fp32_tol(m, n)


def test_batch_argument_errors():
    A = dev(inputs.gaussian(100, 70, 1), torch.float32)
    with pytest.raises(tq.TsqrError):
        tq.Batch([A])  # n > 64

"""The allocation-free entry point tsqr_factor_r_noalloc, through the C ABI.

It exists for callers that cannot call cudaMalloc (code inside another
allocator's callback, framework plugins that own all device memory).  It must
give the same R as tsqr_factor, on consecutive calls that reuse its static
scratch, and refuse problems too large for that scratch.  This file is
collected last so that a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

from conftest import assert_colwise_close, fp64_tol
from paper_0808_2664_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_0808_2664_gb300 as tq  # noqa: E402
from paper_0808_2664_gb300._lib import lib  # noqa: E402


def _dev(A):
    return tq.as_colmajor(torch.from_numpy(np.asfortranarray(A)).to("cuda"))


def _noalloc_r(A):
    m, n = A.shape
    Ad = _dev(A)
    R = tq.colmajor(n, n, torch.float64)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib().tsqr_factor_r_noalloc(m, n, ctypes.c_void_p(Ad.data_ptr()), Ad.stride(1),
                                      ctypes.c_void_p(R.data_ptr()), R.stride(1), stream)
    assert rc == 0, lib().tsqr_status_string(rc)
    torch.cuda.synchronize()
    return R.cpu().numpy()


@pytest.mark.parametrize("m,n", [(20000, 64), (4096, 32), (1000, 7), (80000, 64)])
def test_noalloc_matches_tsqr_factor_twice(m, n):
    for seed in (11, 12):  # two calls in a row reuse the same scratch
        A = inputs.gaussian(m, n, seed)
        R_ref, _ = tq.tsqr_factor(_dev(A), keep_q=False)
        R = _noalloc_r(A)
        ref = R_ref.cpu().numpy()
        assert np.linalg.norm(R - ref) / np.linalg.norm(ref) <= fp64_tol(m, n)
        assert np.array_equal(R, np.triu(R))


@pytest.mark.parametrize("m,n", [(3000, 16), (1_300_000, 4)])
def test_noalloc_matches_oracle(oracle_mod, m, n):
    """Entry by entry against the CPU oracle's R; the second shape has 1270 leaves of
    1024 rows, so its first tree level runs hundreds of nodes."""
    A = inputs.gaussian(m, n, 13)
    _, Ro = oracle_mod.qr(A, want_q=False)
    R = _noalloc_r(A)
    assert np.all(np.diag(R) >= 0)
    assert_colwise_close(R, Ro, fp64_tol(m, n) * np.linalg.cond(Ro), "R")


def test_noalloc_rejects_wide():
    A = torch.zeros((80, 4000), dtype=torch.float64, device="cuda").t()
    R = tq.colmajor(80, 80, torch.float64)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib().tsqr_factor_r_noalloc(4000, 80, ctypes.c_void_p(A.data_ptr()), 4000, ctypes.c_void_p(R.data_ptr()),
                                      80, stream)
    assert rc == 5  # TSQR_ERR_UNSUPPORTED: n > 64


def test_noalloc_rejects_too_large():
    m, n = 1 << 20, 64
    A = torch.zeros((n, m), dtype=torch.float64, device="cuda").t()
    R = tq.colmajor(n, n, torch.float64)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib().tsqr_factor_r_noalloc(m, n, ctypes.c_void_p(A.data_ptr()), m, ctypes.c_void_p(R.data_ptr()), n, stream)
    assert rc == 7  # TSQR_ERR_TOO_LARGE
    assert b"static scratch" in lib().tsqr_status_string(rc)

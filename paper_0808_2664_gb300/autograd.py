"""Differentiable TSQR: torch.autograd.Function over the C-ABI kernels.

Forward: TSQR (n <= 64 in FP64, n <= 128 in FP32) or, for wider FP64
matrices, CAQR with 64-column panels; returns the thin Q and R with
diag(R) >= 0.  Backward: tsqr_qr_backward on the device,
    dA = (dQ + Q copyltu(R dR^T - dQ^T Q)) R^{-T}.
With ``recompute=True`` only A is saved and the factorisation is recomputed
in the backward pass (less memory: no m x n Q kept alive between passes).
"""
from __future__ import annotations

import ctypes

import torch

from . import PREC_FP32, PREC_FP64, as_colmajor, caqr_factor, colmajor, tsqr_factor
from ._lib import TsqrError, check, lib


def _stream(t):
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def _finish(q, where: str) -> None:
    """Reads the handle's device status (a non-finite column norm or pivot,
    a bounded wait that gave up) before freeing it; raises on a nonzero one."""
    st = q.sync_status()
    q.destroy()
    if st != 0:
        raise TsqrError(st, where)


def qr_forward(A: torch.Tensor):
    """(Q, R) of the m x n CUDA tensor A (A itself is not modified).

    Raises TsqrError when the factorisation met a non-finite value."""
    m, n = A.shape
    W = as_colmajor(A.detach()).clone(memory_format=torch.preserve_format)
    W = as_colmajor(W)
    if A.dtype == torch.float64 and n > 64:
        q = caqr_factor(W, b=64)
        R = torch.triu(W[:n, :n]).t().contiguous().t()
        Q = q.form_q()
        _finish(q, "qr_forward (caqr)")
        return Q, R
    R, q = tsqr_factor(W)
    Q = q.form_q()
    _finish(q, "qr_forward (tsqr)")
    return Q, R


def qr_backward(Q, R, dQ, dR):
    """dA of the thin-QR adjoint on the device (FP64 or FP32)."""
    m, n = Q.shape
    prec = PREC_FP64 if Q.dtype == torch.float64 else PREC_FP32
    Q, R, dQ, dR = (as_colmajor(t) for t in (Q, R, dQ, dR))
    dA = colmajor(m, n, Q.dtype, Q.device)
    check(lib().tsqr_qr_backward(m, n, prec, ctypes.c_void_p(Q.data_ptr()), Q.stride(1) if n > 1 else m,
                                 ctypes.c_void_p(R.data_ptr()), R.stride(1) if n > 1 else n,
                                 ctypes.c_void_p(dQ.data_ptr()), dQ.stride(1) if n > 1 else m,
                                 ctypes.c_void_p(dR.data_ptr()), dR.stride(1) if n > 1 else n,
                                 ctypes.c_void_p(dA.data_ptr()), dA.stride(1) if n > 1 else m, None, _stream(Q)),
          "tsqr_qr_backward")
    return dA


class TSQRFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, recompute=False):
        Q, R = qr_forward(A)
        ctx.recompute = bool(recompute)
        if ctx.recompute:
            ctx.save_for_backward(A)
        else:
            ctx.save_for_backward(Q, R)
        return Q, R

    @staticmethod
    def backward(ctx, dQ, dR):
        if ctx.recompute:
            (A,) = ctx.saved_tensors
            Q, R = qr_forward(A)
        else:
            Q, R = ctx.saved_tensors
        m, n = Q.shape
        if dQ is None:
            dQ = torch.zeros_like(Q)
        if dR is None:
            dR = torch.zeros((n, n), dtype=Q.dtype, device=Q.device)
        dA = qr_backward(Q, R, as_colmajor(dQ), as_colmajor(torch.triu(dR)))
        return dA, None


def qr(A: torch.Tensor, recompute: bool = False):
    """Differentiable thin QR (Q, R) of the m x n CUDA tensor A, diag(R) >= 0."""
    return TSQRFunction.apply(A, recompute)

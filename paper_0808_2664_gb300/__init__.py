"""GB300 TSQR / CAQR: Python binding of libtsqr_gb300.so (include/tsqr.h).

The binding only marshals arguments: torch supplies device memory and the
current CUDA stream, every step of the factorisation runs in the library's
CUDA kernels.  Matrices are column-major torch tensors of shape (m, n) with
stride (1, ld), ld >= m -- e.g. ``colmajor(m, n)`` or ``X.t().contiguous().t()``.

    R, q = tsqr_factor(A)          # A is overwritten by the leaf reflectors
    Q = q.form_q()                 # thin Q, A = Q R, diag(R) >= 0
    q.apply_qt(C)                  # C <- Q^T C in place
"""
from __future__ import annotations

import ctypes

from ._lib import TsqrBatchOpts, TsqrError, TsqrOpts, check, lib

__all__ = [
    "TsqrError", "QTree", "CaqrQ", "colmajor", "as_colmajor", "tsqr_factor", "tsqr_q_create",
    "caqr_factor", "caqr_q_create", "Batch", "PREC_FP64", "PREC_FP32", "UPDATE_BF16X3", "UPDATE_TF32X3", "FLAG_APPLY_TF32X3", "FLAG_APPLY_BF16X3", "FLAG_HYBRID_TREE", "FLAG_FLAT_TREE", "FLAG_RECURSIVE_LEAF", "lstsq", "solve_r", "column_norms",
]

PREC_FP64 = 0
PREC_FP32 = 1
UPDATE_BF16X3 = 2
UPDATE_TF32X3 = 3


def _torch():
    import torch

    return torch


def colmajor(m: int, n: int, dtype=None, device="cuda"):
    """Uninitialised m x n column-major tensor (shape (m, n), stride (1, m))."""
    torch = _torch()
    return torch.empty((n, m), dtype=dtype or torch.float64, device=device).t()


def as_colmajor(t):
    """Column-major copy of a 2-D tensor (no copy if already column-major)."""
    if t.dim() == 2 and t.stride(0) == 1 and t.stride(1) >= t.shape[0]:
        return t
    return t.t().contiguous().t()


def _ld(t, name: str, host: bool = False) -> int:
    if t.dim() != 2:
        raise ValueError(f"{name} must be 2-D")
    m, n = t.shape
    if t.is_cuda == host:
        raise ValueError(f"{name} must be a {'host' if host else 'CUDA'} tensor")
    if n <= 1:
        if m > 1 and n == 1 and t.stride(0) != 1:
            raise ValueError(f"{name} must be column-major (unit row stride)")
        return max(1, m, t.stride(1) if n == 1 else m)
    if t.stride(0) != 1 or t.stride(1) < m:
        raise ValueError(f"{name} must be column-major (stride (1, ld) with ld >= {m}); use as_colmajor()")
    return t.stride(1)


def _prec(dtype) -> int:
    torch = _torch()
    if dtype == torch.float64:
        return PREC_FP64
    if dtype == torch.float32:
        return PREC_FP32
    raise TypeError(f"unsupported dtype {dtype}: float64 or float32")


def _stream(t):
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


FLAG_APPLY_BF16X3 = 1
FLAG_HYBRID_TREE = 2
FLAG_FLAT_TREE = 4
FLAG_RECURSIVE_LEAF = 8
FLAG_APPLY_TF32X3 = 16


def _opts(leaf_rows: int, arity: int, flags: int = 0):
    return TsqrOpts(int(leaf_rows), int(arity), int(flags))


class QTree:
    """Handle of a TSQR factorisation: Q as per-level orthogonal factors (Section 2.1).

    Holds a reference to the factored matrix, whose storage keeps the leaf
    Householder vectors.
    """

    def __init__(self, ptr, m: int, n: int, dtype, A=None):
        self._ptr = ptr
        self.m, self.n, self.dtype = m, n, dtype
        self.A = A

    @property
    def ptr(self):
        if not self._ptr:
            raise RuntimeError("handle already destroyed")
        return self._ptr

    def info(self) -> dict:
        m, n, lv, h = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        p, q, lev = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        check(lib().tsqr_q_info(self.ptr, ctypes.byref(m), ctypes.byref(n), ctypes.byref(p), ctypes.byref(lv),
                                ctypes.byref(h), ctypes.byref(q), ctypes.byref(lev)), "tsqr_q_info")
        return {"m": m.value, "n": n.value, "precision": p.value, "leaves": lv.value, "leaf_rows": h.value,
                "arity": q.value, "levels": lev.value}

    def chains(self) -> dict:
        """Leaves per chain and chain count (hybrid / flat trees; 1 and the leaf count otherwise)."""
        L, c = ctypes.c_int64(), ctypes.c_int64()
        check(lib().tsqr_q_chains(self.ptr, ctypes.byref(L), ctypes.byref(c)), "tsqr_q_chains")
        return {"leaves_per_chain": L.value, "chains": c.value}

    def refactor(self, A, R=None):
        """Factor a new matrix of the handle's shape; no allocation.  Returns R."""
        if tuple(A.shape) != (self.m, self.n) or A.dtype != self.dtype:
            raise ValueError("A does not match the handle's shape / dtype")
        lda = _ld(A, "A")
        if R is None:
            R = colmajor(self.n, self.n, self.dtype, A.device)
        ldr = _ld(R, "R")
        check(lib().tsqr_refactor(self.ptr, ctypes.c_void_p(A.data_ptr()), lda, ctypes.c_void_p(R.data_ptr()), ldr,
                                  _stream(A)), "tsqr_refactor")
        self.A = A
        return R

    def _apply(self, fn, C, name):
        if C.dtype != self.dtype or C.shape[0] != self.m:
            raise ValueError(f"C must be {self.m} x k of dtype {self.dtype}")
        ldc = _ld(C, "C")
        check(fn(self.ptr, C.shape[1], ctypes.c_void_p(C.data_ptr()), ldc, _stream(C)), name)
        return C

    def apply_qt(self, C):
        """C <- Q^T C in place (square Q); returns C."""
        return self._apply(lib().tsqr_apply_qt, C, "tsqr_apply_qt")

    def apply_q(self, C):
        """C <- Q C in place (square Q); returns C."""
        return self._apply(lib().tsqr_apply_q, C, "tsqr_apply_q")

    def form_q(self, Q=None):
        """Thin Q (m x n, column-major) including the sign vector."""
        if Q is None:
            Q = colmajor(self.m, self.n, self.dtype, self.A.device if self.A is not None else "cuda")
        ldq = _ld(Q, "Q")
        check(lib().tsqr_form_q(self.ptr, ctypes.c_void_p(Q.data_ptr()), ldq, _stream(Q)), "tsqr_form_q")
        return Q

    def form_q_mul(self, X, Q=None):
        """Q_thin X (m x k) for the n x k column-major CUDA matrix X (tsqr_form_q_mul)."""
        if X.dtype != self.dtype or X.shape[0] != self.n:
            raise ValueError(f"X must be {self.n} x k of dtype {self.dtype}")
        k = X.shape[1]
        if Q is None:
            Q = colmajor(self.m, k, self.dtype, X.device)
        check(lib().tsqr_form_q_mul(self.ptr, k, ctypes.c_void_p(X.data_ptr()), _ld(X, "X"),
                                    ctypes.c_void_p(Q.data_ptr()), _ld(Q, "Q"), _stream(Q)), "tsqr_form_q_mul")
        return Q

    def factor_form_host(self, A_host, Q_host, R_host, A, Q, R):
        """QR of a host matrix with Q and R written back to host memory (tsqr_factor_form_host).
        A_host, Q_host, R_host: column-major CPU tensors; pinned ones are read and written by
        the kernels themselves, pageable ones go through copies.  A, R: device tensors of the
        same shapes; Q: a device tensor, or None to have Q stored straight into a pinned
        Q_host.  Asynchronous on the current stream of A's device."""
        if tuple(A_host.shape) != (self.m, self.n) or A_host.dtype != self.dtype:
            raise ValueError("A_host does not match the handle's shape / dtype")
        check(lib().tsqr_factor_form_host(
            self.ptr, ctypes.c_void_p(A_host.data_ptr()), _ld(A_host, "A_host", host=True),
            ctypes.c_void_p(Q_host.data_ptr()), _ld(Q_host, "Q_host", host=True),
            ctypes.c_void_p(R_host.data_ptr()), _ld(R_host, "R_host", host=True),
            ctypes.c_void_p(A.data_ptr()), _ld(A, "A"),
            ctypes.c_void_p(Q.data_ptr() if Q is not None else None), _ld(Q, "Q") if Q is not None else 0,
            ctypes.c_void_p(R.data_ptr()), _ld(R, "R"), _stream(A)), "tsqr_factor_form_host")
        self.A = A
        return Q_host, R_host

    def lstsq(self, R, B, X=None, rnorm: bool = True):
        """Least-squares solutions of the factored A for the columns of B (tsqr_lstsq).

        R: the n x n R of this factorisation; B: m x k column-major, overwritten
        by Q^T B.  Returns (X, residual norms or None), X n x k."""
        torch = _torch()
        if B.dtype != self.dtype or B.shape[0] != self.m:
            raise ValueError(f"B must be {self.m} x k of dtype {self.dtype}")
        k = B.shape[1]
        if X is None:
            X = colmajor(self.n, k, self.dtype, B.device)
        rn = torch.empty(k, dtype=self.dtype, device=B.device) if rnorm else None
        check(lib().tsqr_lstsq(self.ptr, ctypes.c_void_p(R.data_ptr()), _ld(R, "R"), k,
                               ctypes.c_void_p(B.data_ptr()), _ld(B, "B"), ctypes.c_void_p(X.data_ptr()),
                               _ld(X, "X"), ctypes.c_void_p(rn.data_ptr()) if rn is not None else None, _stream(B)),
              "tsqr_lstsq")
        return X, rn

    PARTS = {"R": 0, "T": 1, "tau": 2, "Y": 3}

    def part(self, what: str, level: int, index: int):
        """A stored factor of leaf (level 0) or tree node `index` (tsqr_q_part): "R" or "T"
        (n x n, column-major), "tau" (n) or, for tree levels, "Y" ((q-1) x n x n blocks)."""
        torch = _torch()
        n = self.n
        dev = self.A.device if self.A is not None else "cuda"
        if what == "tau":
            out = torch.empty(n, dtype=self.dtype, device=dev)
        elif what == "Y":
            q = self.info()["arity"]
            out = torch.empty((q - 1, n, n), dtype=self.dtype, device=dev)
        else:
            out = torch.empty((n, n), dtype=self.dtype, device=dev)
        check(lib().tsqr_q_part(self.ptr, self.PARTS[what], level, index, ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)), "tsqr_q_part")
        if what == "Y":
            return out.transpose(1, 2)  # each block column-major
        return out if what == "tau" else out.t()

    STAGES = ("leaf_factor", "tree_factor", "leaf_apply", "tree_apply")

    def set_timing(self, enable: bool = True) -> None:
        """Record CUDA events around each stage of later calls (clears totals when enabling)."""
        check(lib().tsqr_q_set_timing(self.ptr, 1 if enable else 0), "tsqr_q_set_timing")

    def stage_times(self) -> dict:
        """{stage: (total ms, kernel launches)} since timing was enabled (waits for the events)."""
        ms = (ctypes.c_double * 4)()
        nl = (ctypes.c_int64 * 4)()
        check(lib().tsqr_q_stage_times(self.ptr, ms, nl, 4), "tsqr_q_stage_times")
        return {name: (ms[i], nl[i]) for i, name in enumerate(self.STAGES)}

    def sync_status(self) -> int:
        """Wait for queued work and return the device status code (0 = ok)."""
        torch = _torch()
        return lib().tsqr_sync_status(self.ptr, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))

    def destroy(self):
        if self._ptr:
            lib().tsqr_q_destroy(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def tsqr_q_create(m: int, n: int, dtype=None, device="cuda", leaf_rows: int = 0, arity: int = 0,
                  flags: int = 0) -> QTree:
    """Plan and allocate a handle for m x n problems; factor with QTree.refactor.

    flags: FLAG_APPLY_BF16X3 runs the leaf stage of apply_qt on the tensor
    cores as three BF16 products (float32 handles, n <= 64)."""
    torch = _torch()
    dtype = dtype or torch.float64
    h = ctypes.c_void_p()
    o = _opts(leaf_rows, arity, flags)
    check(lib().tsqr_q_create(m, n, _prec(dtype), ctypes.byref(o), ctypes.byref(h),
                              ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)), "tsqr_q_create")
    return QTree(h, m, n, dtype)


def tsqr_factor(A, R=None, leaf_rows: int = 0, arity: int = 0, keep_q: bool = True, flags: int = 0):
    """TSQR of the column-major m x n CUDA tensor A (overwritten).  Returns (R, QTree or None)."""
    m, n = A.shape
    lda = _ld(A, "A")
    if R is None:
        R = colmajor(n, n, A.dtype, A.device)
    ldr = _ld(R, "R")
    h = ctypes.c_void_p()
    o = _opts(leaf_rows, arity, flags)
    fn = lib().tsqr_factor if _prec(A.dtype) == PREC_FP64 else lib().tsqr_factor_f32
    check(fn(m, n, ctypes.c_void_p(A.data_ptr()), lda, ctypes.c_void_p(R.data_ptr()), ldr, ctypes.byref(o),
             ctypes.byref(h) if keep_q else None, _stream(A)), "tsqr_factor")
    return R, (QTree(h, m, n, A.dtype, A) if keep_q and h.value else None)


def solve_r(R, X):
    """X <- R^{-1} X on the device (R upper triangular n x n, X n x k, column-major); returns X."""
    n, k = X.shape
    check(lib().tsqr_solve_r(n, k, _prec(X.dtype), ctypes.c_void_p(R.data_ptr()), _ld(R, "R"),
                             ctypes.c_void_p(X.data_ptr()), _ld(X, "X"), None, _stream(X)), "tsqr_solve_r")
    return X


def column_norms(B):
    """2-norms of the columns of the column-major CUDA matrix B, computed on the device."""
    torch = _torch()
    m, k = B.shape
    out = torch.empty(k, dtype=B.dtype, device=B.device)
    check(lib().tsqr_column_norms(m, k, _prec(B.dtype), ctypes.c_void_p(B.data_ptr()), _ld(B, "B"),
                                  ctypes.c_void_p(out.data_ptr()), _stream(B)), "tsqr_column_norms")
    return out


def lstsq(A, B, adjoined: bool = False, leaf_rows: int = 0, arity: int = 0):
    """Least squares min ||A X - B|| for the m x n CUDA matrix A and m x k B (neither modified).

    adjoined=False factors A, applies the Q-tree to B and solves with R;
    adjoined=True is the R-only variant Section 1 mentions: TSQR of [A, B]
    keeps only R = [R11, R12; 0, R22], X = R11^{-1} R12, and the residual
    norms are the column norms of R22 (needs n + k within TSQR's width).
    Returns (X, residual norms)."""
    torch = _torch()
    m, n = A.shape
    k = B.shape[1]
    if adjoined:
        W = colmajor(m, n + k, A.dtype, A.device)
        W[:, :n] = A
        W[:, n:] = B
        R, _ = tsqr_factor(W, leaf_rows=leaf_rows, arity=arity, keep_q=False)
        X = colmajor(n, k, A.dtype, A.device).copy_(R[:n, n:])
        solve_r(R[:n, :n], X)
        R22 = colmajor(k, k, A.dtype, A.device).copy_(R[n:, n:])
        return X, column_norms(R22)
    W = as_colmajor(A.detach().clone())
    W = as_colmajor(W)
    R, q = tsqr_factor(W, leaf_rows=leaf_rows, arity=arity)
    Bc = colmajor(m, k, B.dtype, B.device).copy_(B)
    X, rn = q.lstsq(R, Bc)
    st = q.sync_status()
    q.destroy()
    if st != 0:
        raise TsqrError(st, "lstsq")
    return X, rn


class CaqrQ:
    """Handle of a CAQR factorisation: one Q-tree per panel (Section 3)."""

    def __init__(self, ptr, m: int, n: int, dtype, A):
        self._ptr, self.m, self.n, self.dtype, self.A = ptr, m, n, dtype, A

    @property
    def ptr(self):
        if not self._ptr:
            raise RuntimeError("handle already destroyed")
        return self._ptr

    def _apply(self, fn, C, name):
        if C.dtype != self.dtype or C.shape[0] != self.m:
            raise ValueError(f"C must be {self.m} x k of dtype {self.dtype}")
        check(fn(self.ptr, C.shape[1], ctypes.c_void_p(C.data_ptr()), _ld(C, "C"), _stream(C)), name)
        return C

    def apply_qt(self, C):
        return self._apply(lib().caqr_apply_qt, C, "caqr_apply_qt")

    def apply_q(self, C):
        return self._apply(lib().caqr_apply_q, C, "caqr_apply_q")

    def form_q(self, Q=None):
        if Q is None:
            Q = colmajor(self.m, self.n, self.dtype, self.A.device)
        check(lib().caqr_form_q(self.ptr, ctypes.c_void_p(Q.data_ptr()), _ld(Q, "Q"), _stream(Q)), "caqr_form_q")
        return Q

    def set_timing(self, enable: bool = True) -> None:
        check(lib().caqr_q_set_timing(self.ptr, 1 if enable else 0), "caqr_q_set_timing")

    def stage_times(self) -> dict:
        ms = (ctypes.c_double * 4)()
        nl = (ctypes.c_int64 * 4)()
        check(lib().caqr_q_stage_times(self.ptr, ms, nl, 4), "caqr_q_stage_times")
        return {name: (ms[i], nl[i]) for i, name in enumerate(QTree.STAGES)}

    def refactor(self, A):
        """Factor a new m x n matrix in place with the planned workspace (no allocation)."""
        if tuple(A.shape) != (self.m, self.n) or A.dtype != self.dtype:
            raise ValueError("A does not match the handle's shape / dtype")
        check(lib().caqr_refactor(self.ptr, ctypes.c_void_p(A.data_ptr()), _ld(A, "A"), _stream(A)), "caqr_refactor")
        self.A = A
        return A

    def sync_status(self) -> int:
        torch = _torch()
        return lib().caqr_sync_status(self.ptr, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))

    def destroy(self):
        if self._ptr:
            lib().caqr_q_destroy(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def caqr_q_create(m: int, n: int, b: int = 64, dtype=None, device="cuda", update_precision: int = PREC_FP64,
                  leaf_rows: int = 0, arity: int = 0) -> CaqrQ:
    """Plan and allocate a CAQR handle; factor with CaqrQ.refactor."""
    torch = _torch()
    dtype = dtype or torch.float64
    if dtype == torch.float32 and update_precision == PREC_FP64:
        update_precision = PREC_FP32
    h = ctypes.c_void_p()
    o = _opts(leaf_rows, arity)
    check(lib().caqr_q_create(m, n, b, update_precision, ctypes.byref(o), ctypes.byref(h),
                              ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)), "caqr_q_create")
    return CaqrQ(h, m, n, dtype, None)


def caqr_factor(A, b: int = 64, update_precision=None, leaf_rows: int = 0, arity: int = 0,
                keep_q: bool = True):
    """CAQR of the column-major m x n CUDA tensor A in place: R lands in A's upper triangle.

    float64 tensors use the FP64 path; float32 tensors use FP32 storage with
    FP64 reflector generation and, for their trailing updates, FP32 products
    (``PREC_FP32``, default) or three BF16 tensor-core products (``UPDATE_BF16X3``).
    """
    torch = _torch()
    m, n = A.shape
    h = ctypes.c_void_p()
    o = _opts(leaf_rows, arity)
    if A.dtype == torch.float64:
        upd = PREC_FP64 if update_precision is None else update_precision
        fn = lib().caqr_factor
    else:
        upd = PREC_FP32 if update_precision is None else update_precision
        fn = lib().caqr_factor_f32
    check(fn(m, n, ctypes.c_void_p(A.data_ptr()), _ld(A, "A"), b, upd, ctypes.byref(o),
             ctypes.byref(h) if keep_q else None, _stream(A)), "caqr_factor")
    return CaqrQ(h, m, n, A.dtype, A) if keep_q and h.value else None


class Batch:
    """Batched uneven TSQR bound to a list of column-major CUDA matrices.

    ``factor()`` factors all of them in one persistent kernel launch (replayed
    from a CUDA graph by default); each R lands in ``self.R[i]``.
    """

    def __init__(self, As, Rs=None, tile_kb: int = 0, arity: int = 0, autotune: bool = False):
        torch = _torch()
        if not As:
            raise ValueError("empty batch")
        self.dtype = As[0].dtype
        self.A = list(As)
        cnt = len(As)
        if Rs is None:
            Rs = [colmajor(a.shape[1], a.shape[1], self.dtype, a.device) for a in As]
        self.R = list(Rs)
        m = (ctypes.c_int64 * cnt)(*[a.shape[0] for a in As])
        n = (ctypes.c_int64 * cnt)(*[a.shape[1] for a in As])
        lda = (ctypes.c_int64 * cnt)(*[_ld(a, "A") for a in As])
        ldr = (ctypes.c_int64 * cnt)(*[_ld(r, "R") for r in Rs])
        Ap = (ctypes.c_void_p * cnt)(*[a.data_ptr() for a in As])
        Rp = (ctypes.c_void_p * cnt)(*[r.data_ptr() for r in Rs])
        for a in As:
            if a.dtype != self.dtype:
                raise TypeError("all matrices of a batch share one dtype")
        o = TsqrBatchOpts(int(tile_kb), int(arity), 1 if autotune else 0, 0)
        h = ctypes.c_void_p()
        check(lib().tsqr_batch_create(cnt, m, n, Ap, lda, Rp, ldr, _prec(self.dtype), ctypes.byref(o),
                                      ctypes.byref(h), _stream(As[0])), "tsqr_batch_create")
        self._ptr = h

    @property
    def ptr(self):
        if not self._ptr:
            raise RuntimeError("handle already destroyed")
        return self._ptr

    def factor(self, graph: bool = True):
        fn = lib().tsqr_batch_factor_graph if graph else lib().tsqr_batch_factor
        check(fn(self.ptr, _stream(self.A[0])), "tsqr_batch_factor")
        return self.R

    def info(self) -> dict:
        kb, q, it, ws = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
        check(lib().tsqr_batch_info(self.ptr, ctypes.byref(kb), ctypes.byref(q), ctypes.byref(it), ctypes.byref(ws)),
              "tsqr_batch_info")
        return {"tile_kb": kb.value, "arity": q.value, "items": it.value, "workspace_bytes": ws.value}

    def sync_status(self) -> int:
        return lib().tsqr_batch_sync_status(self.ptr, _stream(self.A[0]))

    def destroy(self):
        if self._ptr:
            lib().tsqr_batch_destroy(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

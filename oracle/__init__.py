"""CPU oracle for TSQR / CAQR: plain unblocked FP64 Householder QR in C.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline leg may import this package.  The product library
(``paper_0808_2664_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``householder.c`` (compiled with ``-O2
-ffp-contract=off``); this module only builds it and marshals numpy arrays.
Every array is column-major float64 (``numpy.asfortranarray``).

What each function computes, and the paper passage it follows:

* ``qr(A)`` -- the QR factorisation of A with diag(R) >= 0.  TSQR on any
  reduction tree returns this factorisation (Section 2.1, the uniqueness
  argument after Eq. TSQR_binarytree_4); the oracle computes it with the
  trivial tree, i.e. one Householder reflector per column.
* ``apply_qt`` / ``apply_q`` -- products with the square Q = H_0..H_{n-1} D of
  the same factorisation (Section 2.1: Q kept as a product of orthogonal
  factors, applied rather than multiplied out).
* ``form_q`` -- the thin Q (Section 2.1: Q factors with n columns).
* ``larft`` -- the compact-WY T factor of Schreiber and Van Loan that the
  paper cites for the local QR (Section 2.1, last paragraph).
* ``qr_backward`` -- the QR adjoint for a differentiable TSQR (not in the
  paper; it is the standard adjoint of the sign-normalised thin QR).
* ``lstsq`` -- least-squares solutions and residual norms through the same
  Householder QR (Section 1: the tall-skinny least-squares problem TSQR
  serves): Q^T B, then back substitution with R.

Pins (``tests/test_oracle.py``): closed forms for 2x2 and 3x2 inputs, exact
rational QR of tiny integer matrices, R^T R = A^T A via an independent
Cholesky, LAPACK's QR run as a library, orthogonality and residual bounds,
row-permutation and tree-shape invariance, T against the explicit product of
reflectors, and the adjoint against central finite differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "householder.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

_c_i64 = ctypes.c_int64
_c_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile householder.c into liboracle.so next to it (gcc, OpenMP)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-fopenmp",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i64, dp = _c_i64, _c_dp
            lib.oracle_geqr2.argtypes = [i64, i64, dp, i64, dp]
            lib.oracle_extract_r.argtypes = [i64, dp, i64, dp, dp, i64]
            lib.oracle_apply_qt.argtypes = [i64, i64, dp, i64, dp, dp, i64, dp, i64]
            lib.oracle_apply_q.argtypes = [i64, i64, dp, i64, dp, dp, i64, dp, i64]
            lib.oracle_form_q.argtypes = [i64, i64, dp, i64, dp, dp, dp, i64]
            lib.oracle_larft.argtypes = [i64, i64, dp, i64, dp, dp, i64]
            lib.oracle_qr.argtypes = [i64, i64, dp, i64, dp, i64, dp, dp, dp, i64, dp, i64]
            lib.oracle_qr_backward.argtypes = [i64, i64, dp, dp, dp, dp, dp]
            lib.oracle_lstsq.argtypes = [i64, i64, dp, i64, i64, dp, i64, dp, i64, dp]
            lib.oracle_num_threads.restype = ctypes.c_int
            lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
            lib.oracle_set_num_threads.restype = None
            for f in (lib.oracle_geqr2, lib.oracle_extract_r, lib.oracle_apply_qt, lib.oracle_apply_q,
                      lib.oracle_form_q, lib.oracle_larft, lib.oracle_qr, lib.oracle_qr_backward, lib.oracle_lstsq):
                f.restype = None
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(_c_dp)


class Factorization:
    """Householder factors of one matrix: Y (m x n, reflectors below the
    diagonal, R before sign normalisation on and above it), tau (n), d (n)."""

    def __init__(self, Y: np.ndarray, tau: np.ndarray, d: np.ndarray):
        self.Y, self.tau, self.d = Y, tau, d
        self.m, self.n = Y.shape

    @property
    def R(self) -> np.ndarray:
        return self.d[:, None] * np.triu(self.Y[: self.n, : self.n])


def geqr2(A) -> Factorization:
    """Unblocked Householder QR of A (m >= n) with sign vector d = sign(diag R)."""
    lib = _load()
    Y = _f64(A).copy(order="F")
    m, n = Y.shape
    if m < n:
        raise ValueError("the oracle factors m x n matrices with m >= n")
    tau = np.zeros(n)
    lib.oracle_geqr2(m, n, _p(Y), max(m, 1), _p(tau))
    d = np.where(np.diag(Y)[:n] < 0.0, -1.0, 1.0) if n else np.zeros(0)
    return Factorization(Y, tau, d)


def qr(A, want_q: bool = True):
    """(Q, R) of A with diag(R) >= 0; Q is the thin m x n factor (None if not wanted)."""
    lib = _load()
    A = _f64(A)
    m, n = A.shape
    if m < n:
        raise ValueError("the oracle factors m x n matrices with m >= n")
    Y = np.zeros((m, n), order="F")
    tau, d = np.zeros(n), np.zeros(n)
    R = np.zeros((n, n), order="F")
    Q = np.zeros((m, n), order="F") if want_q else None
    lib.oracle_qr(m, n, _p(A), max(m, 1), _p(Y), max(m, 1), _p(tau), _p(d), _p(R), max(n, 1),
                  _p(Q) if want_q else None, max(m, 1))
    return Q, R


def apply_qt(f: Factorization, C) -> np.ndarray:
    """Q^T C for the square Q = H_0 ... H_{n-1} diag(d, I) of factorisation f."""
    lib = _load()
    C = _f64(C).copy(order="F")
    if C.ndim == 1:
        C = C[:, None]
    k = C.shape[1]
    lib.oracle_apply_qt(f.m, f.n, _p(f.Y), max(f.m, 1), _p(f.tau), _p(f.d), k, _p(C), max(f.m, 1))
    return C


def apply_q(f: Factorization, C) -> np.ndarray:
    """Q C for the square Q of factorisation f."""
    lib = _load()
    C = _f64(C).copy(order="F")
    if C.ndim == 1:
        C = C[:, None]
    k = C.shape[1]
    lib.oracle_apply_q(f.m, f.n, _p(f.Y), max(f.m, 1), _p(f.tau), _p(f.d), k, _p(C), max(f.m, 1))
    return C


def form_q(f: Factorization) -> np.ndarray:
    """Thin Q (m x n) of factorisation f, including the sign vector d."""
    lib = _load()
    Q = np.zeros((f.m, f.n), order="F")
    lib.oracle_form_q(f.m, f.n, _p(f.Y), max(f.m, 1), _p(f.tau), _p(f.d), _p(Q), max(f.m, 1))
    return Q


def larft(f: Factorization) -> np.ndarray:
    """Upper-triangular T with H_0 ... H_{n-1} = I - Y T Y^T (Y unit lower trapezoidal)."""
    lib = _load()
    T = np.zeros((f.n, f.n), order="F")
    lib.oracle_larft(f.m, f.n, _p(f.Y), max(f.m, 1), _p(f.tau), _p(T), max(f.n, 1))
    return T


def unit_lower(f: Factorization) -> np.ndarray:
    """The m x n matrix of Householder vectors with the implicit unit diagonal made explicit."""
    Y = np.tril(f.Y, -1)
    Y[np.arange(f.n), np.arange(f.n)] = 1.0
    return Y


def qr_backward(Q, R, dQ, dR) -> np.ndarray:
    """dA for L = <dQ, Q(A)> + <dR, R(A)> with the sign-normalised thin QR A = QR."""
    lib = _load()
    Q, R, dQ, dR = _f64(Q), _f64(R), _f64(dQ), _f64(dR)
    m, n = Q.shape
    dA = np.zeros((m, n), order="F")
    lib.oracle_qr_backward(m, n, _p(Q), _p(R), _p(dQ), _p(dR), _p(dA))
    return dA


def lstsq(A, B):
    """(X, rnorm): X (n x k) minimises ||A X - B||_F column by column; rnorm[c] = ||A x_c - b_c||_2."""
    lib = _load()
    A = _f64(A)
    B = _f64(B)
    if B.ndim == 1:
        B = B[:, None]
    B = np.asfortranarray(B)
    m, n = A.shape
    k = B.shape[1]
    if B.shape[0] != m or m < n:
        raise ValueError("lstsq needs A m x n with m >= n and B with m rows")
    X = np.zeros((n, k), order="F")
    rn = np.zeros(k)
    lib.oracle_lstsq(m, n, _p(A), max(m, 1), k, _p(B), max(m, 1), _p(X), max(n, 1), _p(rn))
    return X, rn


def num_threads() -> int:
    """OpenMP threads the oracle uses (set OMP_NUM_THREADS before the first call)."""
    return int(_load().oracle_num_threads())


def set_num_threads(nthreads: int) -> None:
    """Sets the OpenMP threads of later oracle calls (timing on one core)."""
    _load().oracle_set_num_threads(int(nthreads))

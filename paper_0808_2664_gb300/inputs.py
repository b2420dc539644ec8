"""Seeded synthetic inputs shaped like the paper's tall-skinny workloads.

This module only draws random matrices; it holds none of the factorisation's
arithmetic, so both the CUDA path and the CPU oracle can be fed from it.
Host generators use numpy's PCG64 (``numpy.random.default_rng(seed)``) and
return column-major float64 arrays; the device generator uses a seeded torch
generator on the GPU for the large benchmark inputs.

Recipes (matrices are m x n, m >= n, column-major):

* ``gaussian``  -- iid N(0, 1) entries.
* ``uniform``   -- iid U[lo, hi] entries (square CAQR input).
* ``ill_conditioned`` -- A = G diag(s) W with G iid N(0, 1), W a random n x n
  orthogonal matrix (numpy's LAPACK QR of an iid N(0, 1) matrix, columns sign
  fixed so the draw is Haar distributed), s_i = cond^(-i/(n-1)).
* ``batched_shapes`` -- for the batched workload: m = round(exp(U[ln m_lo,
  ln m_hi])), n drawn uniformly from a small set.
"""
from __future__ import annotations

import numpy as np


def gaussian(m: int, n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((n, m)).T)


def uniform(m: int, n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.uniform(lo, hi, size=(n, m)).T)


def haar_orthogonal(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((n, n))
    q, r = np.linalg.qr(z)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return np.asfortranarray(q * s[None, :])


def singular_values(n: int, cond: float) -> np.ndarray:
    if n == 1:
        return np.ones(1)
    i = np.arange(n, dtype=np.float64)
    return cond ** (-i / (n - 1))


def ill_conditioned(m: int, n: int, seed: int, cond: float = 1e12) -> np.ndarray:
    G = gaussian(m, n, seed)
    W = haar_orthogonal(n, seed + 7919)
    s = singular_values(n, cond)
    return np.asfortranarray((G * s[None, :]) @ W)


def batched_shapes(count: int, seed: int, m_lo: int = 1024, m_hi: int = 65536, ns=(16, 32, 64)):
    rng = np.random.default_rng(seed)
    ms = np.rint(np.exp(rng.uniform(np.log(m_lo), np.log(m_hi), size=count))).astype(np.int64)
    nn = rng.choice(np.asarray(ns, dtype=np.int64), size=count)
    return [(int(a), int(b)) for a, b in zip(ms, nn)]


def gaussian_device(m: int, n: int, seed: int, dtype=None, device="cuda"):
    """iid N(0, 1) m x n column-major matrix drawn directly on the device.

    Returned as a torch tensor of shape (n, m) whose row c is column c of A
    (i.e. the column-major storage of A), so ``.data_ptr()`` is A with lda = m.
    """
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return torch.randn((n, m), generator=g, dtype=dtype or torch.float64, device=device)

"""TSQR across ranks: one row slab per rank and one exchange of packed R factors.

Section 2.1's reduction tree also runs over processors: each rank factors its
rows (A_p = Q_p R_p), the n x n triangles are exchanged (only the n(n+1)/2
words of each upper triangle travel), and the stacked triangles are factored
again.  Here every rank gathers all P triangles and factors the P*n x n stack
itself, so every rank ends with the same R and no second message is needed
(the redundant, butterfly-style variant of the tree).  The thin Q of the
whole matrix is block-row distributed: rank p holds Q_p * Qtop[p*n:(p+1)*n, :],
formed by applying the local Q-tree to [Qtop block; 0].

The local factorisation is pluggable: by default the CUDA TSQR of this
package (one GPU per rank, NCCL); tests pass a CPU stand-in and use gloo.
"""
from __future__ import annotations

from typing import Callable, Optional, Tuple

import torch
import torch.distributed as dist

# local_qr(A) -> (R, apply_q) where apply_q(X: n x n) returns the m x n product Q_thin X.
LocalQR = Callable[[torch.Tensor], Tuple[torch.Tensor, Callable[[torch.Tensor], torch.Tensor]]]


def _upper_index(n: int, device):
    iu = torch.triu_indices(n, n, device=device)
    order = torch.argsort(iu[1] * n + iu[0])  # column by column
    return iu[:, order]


def pack_upper(R: torch.Tensor) -> torch.Tensor:
    """The n(n+1)/2 entries of the upper triangle of R, column by column."""
    iu = _upper_index(R.shape[0], R.device)
    return R[iu[0], iu[1]].contiguous()


def unpack_upper(v: torch.Tensor, n: int) -> torch.Tensor:
    iu = _upper_index(n, v.device)
    R = torch.zeros((n, n), dtype=v.dtype, device=v.device)
    R[iu[0], iu[1]] = v
    return R


def gpu_local_qr(A: torch.Tensor):
    """Local TSQR (CAQR for FP64 n > 64) on this rank's GPU; apply_q uses the kept Q-tree."""
    from . import as_colmajor, caqr_factor, colmajor, tsqr_factor

    m, n = A.shape
    W = as_colmajor(A.detach().clone())
    W = as_colmajor(W)
    if A.dtype == torch.float64 and n > 64:
        q = caqr_factor(W, b=64)
        R = as_colmajor(torch.triu(W[:n, :n]))
    else:
        R, q = tsqr_factor(W)

    def apply_q(X: torch.Tensor) -> torch.Tensor:
        E = colmajor(m, X.shape[1], A.dtype, A.device)
        E.zero_()
        E[:n, :] = X
        return q.apply_q(E)

    return R, apply_q


def dist_tsqr(A_local: torch.Tensor, group=None, local_qr: Optional[LocalQR] = None, want_q: bool = True):
    """TSQR of the row-distributed matrix [A_0; ...; A_{P-1}] (A_p on rank p, m_p x n, m_p >= n).

    Returns (Q_local, R): R (n x n, diag >= 0) is identical on every rank and
    Q_local is this rank's m_p x n block of the thin Q (None if not wanted).
    """
    local_qr = local_qr or gpu_local_qr
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    n = A_local.shape[1]
    R_p, apply_p = local_qr(A_local)
    packed = pack_upper(R_p)
    gathered = [torch.empty_like(packed) for _ in range(world)]
    dist.all_gather(gathered, packed, group=group)
    stack = torch.cat([unpack_upper(v, n) for v in gathered], dim=0)  # P*n x n, stacked triangles
    R, apply_top = local_qr(stack)
    if not want_q:
        return None, R
    eye = torch.zeros((n, n), dtype=stack.dtype, device=stack.device)
    eye.fill_diagonal_(1.0)
    Q_top = apply_top(eye)                 # thin Q of the stack, P*n x n
    block = Q_top[rank * n:(rank + 1) * n, :]
    return apply_p(block), R

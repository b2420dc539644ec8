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
package (one GPU per rank, NCCL) with the stacked triangles factored by the
structured tree-node kernel; tests pass a CPU stand-in and use gloo.
DistTsqr is the plan-once form (handles and buffers kept across calls).
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
    """Local TSQR (CAQR for FP64 n > 64) on this rank's GPU; apply_q(X) = Q_thin X from the kept Q-tree."""
    from . import as_colmajor, caqr_factor, colmajor, tsqr_factor

    m, n = A.shape
    W = as_colmajor(A.detach().clone())
    W = as_colmajor(W)
    if A.dtype == torch.float64 and n > 64:
        q = caqr_factor(W, b=64)
        R = as_colmajor(torch.triu(W[:n, :n]))

        def apply_q(X: torch.Tensor) -> torch.Tensor:
            E = colmajor(m, X.shape[1], A.dtype, A.device)
            E.zero_()
            E[:n, :] = X
            return q.apply_q(E)

        return R, apply_q
    R, q = tsqr_factor(W)

    def apply_q(X: torch.Tensor) -> torch.Tensor:
        return q.form_q_mul(as_colmajor(X.contiguous()))

    return R, apply_q


def gpu_stack_qr(stack: torch.Tensor):
    """QR of P stacked n x n upper triangles (P n x n) on the GPU: leaves of n rows
    (each already triangular) and one structured tree node of arity P (P <= 16) or a
    4-ary tree above them, so the triangles' zeros are never touched (Section 2.1)."""
    from . import as_colmajor, tsqr_factor

    pn, n = stack.shape
    P = pn // n
    W = as_colmajor(stack.detach().clone())
    W = as_colmajor(W)
    if W.dtype == torch.float64 and n > 64:
        return gpu_local_qr(stack)
    arity = P if 2 <= P <= 16 else 4
    R, q = tsqr_factor(W, leaf_rows=n, arity=arity)

    def apply_q(X: torch.Tensor) -> torch.Tensor:
        return q.form_q_mul(as_colmajor(X.contiguous()))

    return R, apply_q


def dist_tsqr(A_local: torch.Tensor, group=None, local_qr: Optional[LocalQR] = None, want_q: bool = True,
              top_qr: Optional[LocalQR] = None):
    """TSQR of the row-distributed matrix [A_0; ...; A_{P-1}] (A_p on rank p, m_p x n, m_p >= n).

    Returns (Q_local, R): R (n x n, diag >= 0) is identical on every rank and
    Q_local is this rank's m_p x n block of the thin Q (None if not wanted).
    The top of the tree factors the gathered triangles with top_qr (default:
    the structured GPU node kernel when local_qr is the GPU path, local_qr
    otherwise).
    """
    if local_qr is None:
        local_qr = gpu_local_qr
        top_qr = top_qr or gpu_stack_qr
    top_qr = top_qr or local_qr
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    n = A_local.shape[1]
    R_p, apply_p = local_qr(A_local)
    packed = pack_upper(R_p)
    gathered = [torch.empty_like(packed) for _ in range(world)]
    dist.all_gather(gathered, packed, group=group)
    stack = torch.cat([unpack_upper(v, n) for v in gathered], dim=0)  # P*n x n, stacked triangles
    R, apply_top = top_qr(stack)
    if not want_q:
        return None, R
    eye = torch.zeros((n, n), dtype=stack.dtype, device=stack.device)
    eye.fill_diagonal_(1.0)
    Q_top = apply_top(eye)                 # thin Q of the stack, P*n x n
    block = Q_top[rank * n:(rank + 1) * n, :]
    return apply_p(block), R


class DistTsqr:
    """Plan-once parallel TSQR over the ranks of `group` (Section 2.1): each rank
    factors its m_local x n slab with its own Q-tree handle, the packed R
    triangles travel in one all_gather, every rank factors the P stacked
    triangles with the structured tree-node kernel, and each rank forms its
    block of the thin Q as Q_p [Qtop_p; 0].  Handles and buffers are created
    once; factor() allocates nothing on the device but the outputs it is not
    given."""

    def __init__(self, m_local: int, n: int, dtype=torch.float64, device=None, group=None):
        from . import colmajor, tsqr_q_create

        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.m, self.n, self.dtype = m_local, n, dtype
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        P = self.world
        self.local = tsqr_q_create(m_local, n, dtype, self.device)
        self.top = tsqr_q_create(P * n, n, dtype, self.device, leaf_rows=n, arity=P if 2 <= P <= 16 else 4)
        self.R_local = colmajor(n, n, dtype, self.device)
        self.R = colmajor(n, n, dtype, self.device)
        self.stack = colmajor(P * n, n, dtype, self.device)
        npk = n * (n + 1) // 2
        self.gathered = [torch.empty(npk, dtype=dtype, device=self.device) for _ in range(P)]
        self.Qtop = colmajor(P * n, n, dtype, self.device)
        self.iu = _upper_index(n, self.device)

    def factor(self, A_local: torch.Tensor, Q_local: Optional[torch.Tensor] = None):
        """(Q_local, R) of the distributed matrix; A_local is overwritten by its reflectors."""
        from . import as_colmajor

        n = self.n
        self.local.refactor(A_local, self.R_local)
        packed = self.R_local[self.iu[0], self.iu[1]].contiguous()
        dist.all_gather(self.gathered, packed, group=self.group)
        self.stack.zero_()
        for p, v in enumerate(self.gathered):
            blk = self.stack[p * n:(p + 1) * n]
            blk[self.iu[0], self.iu[1]] = v
        self.top.refactor(self.stack, self.R)
        self.top.form_q(self.Qtop)
        X = as_colmajor(self.Qtop[self.rank * n:(self.rank + 1) * n].contiguous())
        Q_local = self.local.form_q_mul(X, Q_local)
        return Q_local, self.R

    def destroy(self):
        self.local.destroy()
        self.top.destroy()

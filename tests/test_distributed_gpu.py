"""Row-slab TSQR across ranks (Section 2.1's parallel TSQR) with the GPU local path.

  * dist_tsqr on a world-size-1 NCCL group: the real all_gather of packed R
    triangles, the structured top-of-tree factorisation and the per-rank Q
    block, against the CPU oracle;
  * P ranks emulated one after another in this process (no collective, no
    kernels waiting on one another): every slab's GPU TSQR, the stacked
    triangles factored by the structured tree-node kernel, each slab's Q block
    formed as Q_p [Qtop_p; 0] with tsqr_form_q_mul -- the whole-matrix R and Q
    against the oracle;
  * tsqr_form_q_mul against the oracle's Q X.
"""
import os
import socket

import numpy as np
import pytest

from conftest import assert_colwise_close, fp64_tol
from paper_0808_2664_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import torch.distributed as dist  # noqa: E402

import paper_0808_2664_gb300 as tq  # noqa: E402
from paper_0808_2664_gb300 import distributed as D  # noqa: E402


def dev(A):
    return tq.as_colmajor(torch.from_numpy(np.asfortranarray(A)).cuda())


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_dist_tsqr_nccl_world_size_one(oracle_mod):
    m, n = 50000, 32
    A = inputs.gaussian(m, n, 4400)
    Qo, Ro = oracle_mod.qr(A)
    os.environ.setdefault("NCCL_NVLS_ENABLE", "0")
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{_free_port()}", rank=0, world_size=1,
                            device_id=torch.device("cuda", 0))
    try:
        Ql, R = D.dist_tsqr(dev(A))
        torch.cuda.synchronize()
    finally:
        dist.destroy_process_group()
    tol = fp64_tol(m, n) * np.linalg.cond(Ro)
    assert_colwise_close(R.cpu().numpy(), Ro, tol, "R")
    assert_colwise_close(Ql.cpu().numpy(), Qo, tol, "Q")


@pytest.mark.parametrize("P,m,n", [(3, 30000, 16), (8, 64000, 64), (20, 40000, 8), (1, 5000, 24)])
def test_emulated_ranks_structured_top(oracle_mod, P, m, n):
    A = inputs.gaussian(m, n, 4500 + P)
    Qo, Ro = oracle_mod.qr(A)
    bounds = np.linspace(0, m, P + 1).astype(int)
    locals_ = [D.gpu_local_qr(dev(A[bounds[p]:bounds[p + 1]])) for p in range(P)]
    stack = torch.cat([torch.triu(r) for r, _ in locals_], dim=0)
    R, apply_top = D.gpu_stack_qr(stack)
    eye = torch.eye(n, dtype=torch.float64, device="cuda")
    Qtop = apply_top(eye)
    Q = torch.cat([locals_[p][1](Qtop[p * n:(p + 1) * n]) for p in range(P)], dim=0)
    torch.cuda.synchronize()
    tol = fp64_tol(m, n) * np.linalg.cond(Ro)
    assert_colwise_close(R.cpu().numpy(), Ro, tol, "R")
    assert_colwise_close(Q.cpu().numpy(), Qo, tol, "Q")


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_form_q_mul_matches_oracle(oracle_mod, dtype):
    m, n, k = 20000, 48, 13
    A = inputs.gaussian(m, n, 4600)
    X = inputs.gaussian(n, k, 4601)
    if dtype == torch.float32:
        A, X = A.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64)
    Qo, _ = oracle_mod.qr(A)
    Ad = tq.as_colmajor(torch.from_numpy(A).to("cuda", dtype))
    _, q = tq.tsqr_factor(Ad, leaf_rows=512)
    QX = q.form_q_mul(tq.as_colmajor(torch.from_numpy(X).to("cuda", dtype))).double().cpu().numpy()
    from conftest import fp32_tol

    tol = (fp64_tol if dtype == torch.float64 else fp32_tol)(m, n)
    assert_colwise_close(QX, Qo @ X, 4 * tol * np.linalg.cond(A), "QX")
    q.destroy()


def test_dist_tsqr_plan_once_nccl(oracle_mod):
    """The plan-once DistTsqr on a world-size-1 NCCL group, two factorisations in a row."""
    m, n = 30000, 64
    os.environ.setdefault("NCCL_NVLS_ENABLE", "0")
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{_free_port()}", rank=0, world_size=1,
                            device_id=torch.device("cuda", 0))
    try:
        dt = D.DistTsqr(m, n, torch.float64)
        for seed in (4700, 4701):
            A = inputs.gaussian(m, n, seed)
            Qo, Ro = oracle_mod.qr(A)
            Ql, R = dt.factor(dev(A))
            torch.cuda.synchronize()
            tol = fp64_tol(m, n) * np.linalg.cond(Ro)
            assert_colwise_close(R.cpu().numpy(), Ro, tol, "R")
            assert_colwise_close(Ql.cpu().numpy(), Qo, tol, "Q")
        dt.destroy()
    finally:
        dist.destroy_process_group()


def test_bench_dist_run_world_size_one():
    """bench.py's row-slab measurement (its path for --gpus N > 1) on a world-size-1 group."""
    import argparse
    import importlib.util

    spec = importlib.util.spec_from_file_location(
        "bench", os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    args = argparse.Namespace(m=65536, n=32, steps=2, warmup=1)
    os.environ.setdefault("NCCL_NVLS_ENABLE", "0")
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{_free_port()}", rank=0, world_size=1,
                            device_id=torch.device("cuda", 0))
    try:
        res = bench.dist_run(tq, torch, dist, args, 0, 1)
    finally:
        dist.destroy_process_group()
    assert res["ms_per_step"] > 0 and res["e2e"]["value"] > 0
    assert res["slab_backward_error"] <= fp64_tol(65536, 32)

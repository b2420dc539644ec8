"""TSQR across ranks (row slabs + one exchange of packed R factors), on CPU with gloo.

Each rank factors its slab with the CPU oracle (a stand-in for the per-GPU
TSQR), the packed triangles are all-gathered, and every rank factors the
stack.  The result must be the QR of the whole matrix.  A second test makes
one rank fail before the exchange and checks that the other gets an error
instead of hanging.
"""
import os
import socket
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _oracle_local_qr(A):
    import oracle

    Q, R = oracle.qr(A.numpy())

    def apply_q(X):
        return torch.from_numpy(Q @ X.numpy())

    return torch.from_numpy(R), apply_q


def _worker(rank, world, port, m_per, n, outdir, fail_rank):
    import sys

    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import datetime

    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    from paper_0808_2664_gb300 import distributed as D
    from paper_0808_2664_gb300 import inputs

    A = inputs.gaussian(m_per * world, n, 777)
    A_loc = torch.from_numpy(np.ascontiguousarray(A[rank * m_per:(rank + 1) * m_per]))
    try:
        if rank == fail_rank:
            raise RuntimeError("injected failure before the exchange")
        Q_loc, R = D.dist_tsqr(A_loc, local_qr=_oracle_local_qr)
        np.save(os.path.join(outdir, f"R{rank}.npy"), R.numpy())
        np.save(os.path.join(outdir, f"Q{rank}.npy"), Q_loc.numpy())
        open(os.path.join(outdir, f"ok{rank}"), "w").close()
    except Exception as e:  # the survivor records the error it saw
        with open(os.path.join(outdir, f"err{rank}"), "w") as f:
            f.write(repr(e))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _run(world, m_per, n, fail_rank=-1):
    outdir = tempfile.mkdtemp()
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, world, port, m_per, n, outdir, fail_rank)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        if p.is_alive():
            p.kill()
            p.join()
    return outdir


@pytest.mark.parametrize("world,m_per,n", [(2, 300, 12), (3, 257, 7)])
def test_dist_tsqr_matches_whole_matrix_qr(world, m_per, n):
    import oracle

    from conftest import fp64_tol
    from paper_0808_2664_gb300 import inputs

    out = _run(world, m_per, n)
    A = inputs.gaussian(m_per * world, n, 777)
    Qo, Ro = oracle.qr(A)
    Rs = [np.load(os.path.join(out, f"R{r}.npy")) for r in range(world)]
    Q = np.vstack([np.load(os.path.join(out, f"Q{r}.npy")) for r in range(world)])
    tol = fp64_tol(A.shape[0], n)
    for R in Rs:
        assert np.array_equal(R, Rs[0])  # every rank factors the same stack
        assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= tol * np.linalg.cond(A)
    assert np.linalg.norm(Q - Qo) <= tol * np.linalg.cond(A) * np.sqrt(n)
    assert np.linalg.norm(A - Q @ Rs[0]) / np.linalg.norm(A) <= tol


def test_pack_unpack_roundtrip():
    from paper_0808_2664_gb300 import distributed as D

    R = torch.triu(torch.randn(9, 9, dtype=torch.float64))
    v = D.pack_upper(R)
    assert v.numel() == 9 * 10 // 2
    assert torch.equal(D.unpack_upper(v, 9), R)
    assert v[0] == R[0, 0] and v[1] == R[0, 1] and v[2] == R[1, 1]  # column by column


def test_failed_rank_is_reported_not_hung():
    out = _run(2, 100, 5, fail_rank=1)
    assert os.path.exists(os.path.join(out, "err1"))
    # The survivor's collective ends with an error (peer gone) within the group timeout.
    assert os.path.exists(os.path.join(out, "err0")) and not os.path.exists(os.path.join(out, "ok0"))

"""QR backward on the device: finite differences, the oracle's adjoint, autograd plumbing."""
import numpy as np
import pytest

from conftest import fp32_tol, fp64_tol
from paper_0808_2664_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_0808_2664_gb300 as tq  # noqa: E402
from paper_0808_2664_gb300 import autograd as tqa  # noqa: E402


def dev(A, dtype=torch.float64):
    return tq.as_colmajor(torch.from_numpy(np.asfortranarray(A)).to("cuda", dtype))


def test_central_finite_differences():
    """L(A) = <dQ, Q(A)> + <dR, R(A)>; central differences with h = 1e-6 in FP64 on 512 x 8."""
    m, n = 512, 8
    A = dev(inputs.gaussian(m, n, 5000)).requires_grad_(True)
    dQ = dev(inputs.gaussian(m, n, 5001))
    dR = dev(np.triu(inputs.gaussian(n, n, 5002)))
    Q, R = tqa.qr(A)
    (torch.sum(dQ * Q) + torch.sum(dR * R)).backward()
    g = A.grad.detach()

    def loss(X):
        q, r = tqa.qr_forward(X)
        return float(torch.sum(dQ * q) + torch.sum(dR * r))

    h = 1e-6
    for s in range(4):
        E = dev(inputs.gaussian(m, n, 6000 + s))
        fd = (loss(A.detach() + h * E) - loss(A.detach() - h * E)) / (2 * h)
        an = float(torch.sum(g * E))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


@pytest.mark.parametrize("m,n,dtype", [(4096, 32, torch.float64), (3000, 128, torch.float64),
                                       (4096, 64, torch.float32), (777, 1, torch.float64)])
def test_backward_matches_oracle(oracle_mod, m, n, dtype):
    A = inputs.gaussian(m, n, 70 + n)
    Qo, Ro = oracle_mod.qr(A)
    dQ = inputs.gaussian(m, n, 71)
    dR = np.triu(inputs.gaussian(n, n, 72))
    dA_o = oracle_mod.qr_backward(Qo, Ro, dQ, np.asfortranarray(dR))
    dA = tqa.qr_backward(dev(Qo, dtype), dev(Ro, dtype), dev(dQ, dtype), dev(dR, dtype)).double().cpu().numpy()
    tol = (fp64_tol if dtype == torch.float64 else fp32_tol)(m, n)
    kappa = np.linalg.cond(Ro)
    assert np.linalg.norm(dA - dA_o) / np.linalg.norm(dA_o) <= tol * kappa


@pytest.mark.parametrize("recompute", [False, True])
def test_autograd_full_chain_matches_oracle(oracle_mod, recompute):
    m, n = 20000, 48
    A_np = inputs.gaussian(m, n, 91)
    A = dev(A_np).requires_grad_(True)
    dQ = inputs.gaussian(m, n, 92)
    dR = inputs.gaussian(n, n, 93)  # full dR: only its upper triangle reaches R
    Q, R = tqa.qr(A, recompute)
    Q.backward(dev(dQ), retain_graph=True)
    g1 = A.grad.clone()
    A.grad = None
    (torch.sum(Q * dev(dQ)) + torch.sum(R * dev(dR))).backward()
    Qo, Ro = oracle_mod.qr(A_np)
    dA_o = oracle_mod.qr_backward(Qo, Ro, dQ, np.asfortranarray(np.triu(dR)))
    got = A.grad.cpu().numpy()
    assert np.linalg.norm(got - dA_o) / np.linalg.norm(dA_o) <= fp64_tol(m, n) * np.linalg.cond(A_np)
    assert torch.isfinite(g1).all()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_full_size_gradient_against_oracle(oracle_mod, dtype):
    """m = 1,048,576 x n = 128: device forward + backward; the oracle's adjoint from the same Q, R."""
    m, n = 1 << 20, 128
    A = inputs.gaussian_device(m, n, 5555, dtype=dtype).t()
    Q, R = tqa.qr_forward(A)
    g = torch.Generator(device="cuda")
    g.manual_seed(5556)
    dQ = torch.randn((n, m), generator=g, dtype=dtype, device="cuda").t()
    dR = torch.triu(torch.randn((n, n), generator=g, dtype=dtype, device="cuda"))
    dA = tqa.qr_backward(Q, R, dQ, tq.as_colmajor(dR))
    # Forward quality in FP64 on the device.
    Q64, R64, A64 = Q.double(), R.double(), A.double()
    tol = (fp64_tol if dtype == torch.float64 else fp32_tol)(m, n)
    assert (torch.linalg.norm(A64 - Q64 @ R64) / torch.linalg.norm(A64)).item() <= tol
    assert torch.linalg.norm(torch.eye(n, dtype=torch.float64, device="cuda") - Q64.t() @ Q64).item() <= tol
    Qh, Rh = Q64.cpu().numpy(), R64.cpu().numpy()
    dA_o = oracle_mod.qr_backward(Qh, Rh, dQ.double().cpu().numpy(), dR.double().t().contiguous().t().cpu().numpy())
    got = dA.double().cpu().numpy()
    assert np.linalg.norm(got - dA_o) / np.linalg.norm(dA_o) <= tol * np.linalg.cond(Rh)


def test_forward_reports_nonfinite():
    """A NaN met by the factorisation is read from the handle's status word and raised."""
    A = inputs.gaussian(2048, 8, 9)
    A[100, 3] = np.nan
    with pytest.raises(tq.TsqrError) as ei:
        tqa.qr_forward(dev(A))
    assert ei.value.code == 4  # TSQR_ERR_NONFINITE

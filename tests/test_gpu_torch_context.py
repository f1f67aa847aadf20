"""The PyTorch-ops DPSR that bench.py times as context (not a product path)
must compute the same layer as the oracle before its time means anything:
chi within 1e-5 and the autograd gradients within 1e-4 of the FP64 oracle."""
import numpy as np
import pytest

from paper_2106_03452_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("r,N,sigma", [(32, 2000, 2.0), (64, 3000, 1.5)])
def test_torch_ops_context_matches_oracle(oracle, r, N, sigma):
    import torch
    import bench
    from gpu_util import relmax
    rng = synth.Rng(3100 + r)
    pts = (rng.uniform(N, 3) * 1.4 - 0.2).astype(np.float32)
    nrm = rng.normal(N, 3).astype(np.float32)
    G = rng.normal(r, r, r).astype(np.float32)
    P = torch.from_numpy(pts).cuda().requires_grad_(True)
    Nn = torch.from_numpy(nrm).cuda().requires_grad_(True)
    chi = bench.torch_ops_dpsr(P, Nn, r, sigma)
    dp, dn = torch.autograd.grad((chi * torch.from_numpy(G).cuda()).sum(), (P, Nn))
    ref = oracle.forward(r, sigma, pts.astype(np.float64), nrm.astype(np.float64))
    rdp, rdn = oracle.backward(r, sigma, pts.astype(np.float64), nrm.astype(np.float64), G.astype(np.float64))
    assert relmax(chi.detach().cpu().numpy(), ref) <= 1e-5
    assert relmax(dn.cpu().numpy(), rdn) <= 1e-4
    assert relmax(dp.cpu().numpy(), rdp) <= 1e-4

"""Helpers of the GPU parity tests: run the CUDA path and the oracle on the
same FP32 inputs and compare."""
import numpy as np
import torch

from paper_2106_03452_gb300.dpsr import Plan


def relmax(a, b):
    """max |a - b| / max |b|."""
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def gpu_fwd_bwd(r, sigma, pts, nrm, dchi=None, plan=None):
    plan = plan or Plan(r, sigma)
    P = torch.from_numpy(np.ascontiguousarray(pts, np.float32)).cuda()
    Nn = torch.from_numpy(np.ascontiguousarray(nrm, np.float32)).cuda()
    chi = plan.forward(P, Nn)
    st = plan.sync()
    out = dict(chi=chi.cpu().numpy(), status=st, plan=plan)
    if st == 0:
        out["scalars"] = plan.scalars()
    if dchi is not None and st == 0:
        G = torch.from_numpy(np.ascontiguousarray(dchi, np.float32)).cuda()
        dp, dn = plan.backward(G)
        out["bstatus"] = plan.sync()
        out["dpoints"], out["dnormals"] = dp.cpu().numpy(), dn.cpu().numpy()
    return out

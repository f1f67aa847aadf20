"""The differentiable loop on top of the DPSR layer: a loss defined on the
indicator at target points, L = mean_k chi(q_k)^2 (zero when the reconstructed
surface passes through the targets), and gradient steps on the oriented point
cloud through the hand-written adjoint (Sec. 3.2 optimises the source cloud
through the solver in the same way; its Chamfer/Marching-Cubes loss is
replaced here by a loss that needs no mesh).

The lookup chi(q) and its adjoint run in libdpsr kernels (dpsr_grid_sample /
dpsr_grid_splat); Adam is PyTorch's optimiser on CUDA tensors.
"""
from __future__ import annotations

import time

import torch

from . import libdpsr as L
from .dpsr import Plan, dpsr


class GridSample(torch.autograd.Function):
    """chi(q): trilinear lookup of an r^3 grid at query points, with the
    rasterization of the incoming gradient as its backward."""

    @staticmethod
    def forward(ctx, chi, q):
        r = chi.shape[0]
        q = q.contiguous()
        out = torch.empty(q.shape[0], device=chi.device, dtype=torch.float32)
        st = torch.cuda.current_stream(chi.device).cuda_stream
        L.dpsr_grid_sample(chi.contiguous().data_ptr(), r, q.data_ptr(), q.shape[0], out.data_ptr(), st)
        ctx.save_for_backward(q)
        ctx.r = r
        return out

    @staticmethod
    def backward(ctx, g):
        (q,) = ctx.saved_tensors
        r = ctx.r
        g = g.contiguous()
        dchi = torch.empty((r, r, r), device=q.device, dtype=torch.float32)
        st = torch.cuda.current_stream(q.device).cuda_stream
        L.dpsr_grid_splat(dchi.data_ptr(), r, q.data_ptr(), g.data_ptr(), q.shape[0], False, st)
        return dchi, None


def surface_loss(chi: torch.Tensor, targets: torch.Tensor) -> torch.Tensor:
    v = GridSample.apply(chi, targets)
    return (v * v).mean()


def optimize(points, normals, targets, r=256, sigma=2.0, steps=50, lr=2e-3 * 0.7 ** 3, plan=None):
    """`steps` Adam steps on (points, normals) of L = mean chi(q)^2. The
    learning rate defaults to the paper's 256^3 level of its coarse-to-fine
    schedule (2e-3 decayed by 0.7 three times, supplementary Sec. B).
    Returns (loss history, points, normals, seconds per step); the time per
    step leaves out the first step, which carries one-time costs (the
    cluster-size autotuner, Adam's state allocation)."""
    plan = plan or Plan(r, sigma, device=points.device, n_max=points.shape[0])
    c = points.detach().clone().requires_grad_(True)
    n = normals.detach().clone().requires_grad_(True)
    opt = torch.optim.Adam([c, n], lr=lr)
    hist = []
    t0 = None
    for k in range(steps):
        if k == 1:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
        opt.zero_grad(set_to_none=False)
        loss = surface_loss(dpsr(c, n, plan), targets)
        loss.backward()
        opt.step()
        hist.append(loss.detach())
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / (steps - 1) if steps > 1 else float("nan")
    return [float(h) for h in hist], c.detach(), n.detach(), dt

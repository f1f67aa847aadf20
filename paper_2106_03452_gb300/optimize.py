"""The optimisation setting of Sec. 3.2 (details in supplementary Sec. B):
surface reconstruction from an unoriented point cloud by optimising an
oriented point cloud through the DPSR layer.

Per iteration: chi = DPSR(points, normals); a mesh at level 0; points drawn
on it by area; the bi-directional L2 Chamfer distance to the input cloud;
its gradient back to the mesh points, through Eq. 6 to chi, and through the
DPSR adjoint to the points and normals; an Adam step. Every `resample`
iterations, and when the grid size grows, the points and normals are
replaced by points drawn uniformly on the largest mesh component (with its
normals). The schedule is coarse to fine: 32^3, 64^3, 128^3 for 1000
iterations each and 256^3 for 200, sigma = 2, 2, 3 and 3 (5 for noisy
inputs), a learning rate of 2e-3 decayed by 0.7 at each level, 20000 points,
starting from a sphere. Every step runs in libdpsr's kernels; PyTorch holds
the tensors and runs Adam.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import libdpsr as L
from .dpsr import Plan, dpsr
from .mesh import MeshPoints, largest_component, sample

PAPER_LEVELS = ((32, 2.0, 1000), (64, 2.0, 1000), (128, 3.0, 1000), (256, 3.0, 200))


class ChamferLoss(torch.autograd.Function):
    """Bi-directional L2 Chamfer distance between a (differentiable) and b
    (dpsr_chamfer: brute-force nearest neighbours in both directions)."""

    @staticmethod
    def forward(ctx, a, b):
        a, b = a.contiguous(), b.contiguous()
        na, nb = a.shape[0], b.shape[0]
        st = torch.cuda.current_stream(a.device).cuda_stream
        ws_idx = torch.empty(na + nb, dtype=torch.int32, device=a.device)
        ws_d2 = torch.empty(na + nb, device=a.device)
        grad = torch.empty_like(a)
        loss = torch.empty(1, dtype=torch.float64, device=a.device)
        L.dpsr_chamfer(a.data_ptr(), na, b.data_ptr(), nb, ws_idx.data_ptr(), ws_d2.data_ptr(), grad.data_ptr(),
                       loss.data_ptr(), st)
        ctx.save_for_backward(grad)
        return loss.to(a.dtype).reshape(())

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return grad * g, None


def chamfer(a, b):
    return ChamferLoss.apply(a, b)


def sphere_cloud(n: int, radius: float = 0.3, device="cuda", seed: int = 0):
    """n points on a sphere around the cube's centre with outward unit
    normals (a Fibonacci spiral: deterministic and nearly uniform)."""
    k = torch.arange(n, dtype=torch.float64, device=device)
    z = 1.0 - (2.0 * k + 1.0) / n
    rho = torch.sqrt(1.0 - z * z)
    phi = k * (math.pi * (3.0 - math.sqrt(5.0))) + seed
    d = torch.stack([rho * torch.cos(phi), rho * torch.sin(phi), z], 1)
    return (0.5 + radius * d).float(), d.float()


def resample_from(chi, n: int, seed: int):
    """n points and normals drawn uniformly on the largest mesh component."""
    tris, nrm = largest_component(chi.detach())
    if tris.shape[0] == 0:
        raise RuntimeError("empty mesh: nothing to resample")
    return sample(tris, nrm, n, seed)


def _settings(levels, n_points, samples, lr0, decay, resample, seed):
    return np.array([float(x) for lv in levels for x in lv] + [n_points, samples, lr0, decay, resample, seed],
                    np.float64)


def save_checkpoint(path, level, c, n, chi, hist, settings):
    """The state at a level boundary: the next level starts from it exactly
    (its points are drawn from chi's mesh and its Adam state is fresh)."""
    np.savez(path, level=np.int64(level), points=c.detach().cpu().numpy(), normals=n.detach().cpu().numpy(),
             chi=chi.detach().cpu().numpy(), hist=np.array(hist, np.float64).reshape(-1, 6), settings=settings)


def load_checkpoint(path, device):
    z = np.load(path)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
    hist = [tuple(row) for row in z["hist"].tolist()]
    hist = [(int(h[0]), h[1], int(h[2]), h[3], h[4], h[5]) for h in hist]
    return int(z["level"]), t(z["points"]), t(z["normals"]), t(z["chi"]), hist, z["settings"]


def reconstruct(target: torch.Tensor, levels=PAPER_LEVELS, n_points: int = 20000, samples: int = 20000,
                lr0: float = 2e-3, decay: float = 0.7, resample: int = 200, seed: int = 0, log=None,
                checkpoint: str | None = None, resume: str | None = None):
    """Optimise an oriented cloud whose surface fits the unoriented `target`
    cloud (M x 3, CUDA). Returns (points, normals, history) where history
    lists per level (r, sigma, iterations, first loss, last loss, seconds).
    checkpoint: a .npz path written after every completed level (points,
    normals, chi, history); resume: such a file, whose completed levels are
    skipped (the schedule and settings must be the ones it was written with)."""
    settings = _settings(levels, n_points, samples, lr0, decay, resample, seed)
    c, n = sphere_cloud(n_points, device=target.device)
    hist = []
    chi = None
    start = 0
    if resume is not None:
        start, c, n, chi, hist, saved = load_checkpoint(resume, target.device)
        if saved.shape != settings.shape or not np.array_equal(saved, settings):
            raise ValueError("checkpoint was written with another schedule or other settings")
    for li, (r, sigma, iters) in enumerate(levels):
        if li < start:
            continue
        if chi is not None:  # a new grid size starts from the previous level's mesh
            c, n = resample_from(chi, n_points, seed + 7919 * li)
        plan = Plan(r, sigma, device=target.device, n_max=n_points)
        c = c.detach().clone().requires_grad_(True)
        n = n.detach().clone().requires_grad_(True)
        opt = torch.optim.Adam([c, n], lr=lr0 * decay ** li)
        first = last = None
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for it in range(iters):
            if it > 0 and it % resample == 0:
                c2, n2 = resample_from(chi, n_points, seed + 104729 * li + it)
                with torch.no_grad():
                    c.copy_(c2)
                    n.copy_(n2)
                opt = torch.optim.Adam([c, n], lr=lr0 * decay ** li)
            opt.zero_grad(set_to_none=False)
            chi = dpsr(c, n, plan)
            p, _ = MeshPoints.apply(chi, 0.0, samples, seed + 31 * it + 100003 * li)
            loss = chamfer(p, target)
            loss.backward()
            opt.step()
            v = float(loss.detach())
            first = v if first is None else first
            last = v
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        hist.append((r, sigma, iters, first, last, dt))
        if log:
            log(f"level r={r} sigma={sigma}: {iters} iterations, Chamfer {first:.3e} -> {last:.3e}, {dt:.2f} s")
        plan.close()
        chi = chi.detach()
        if checkpoint is not None:
            save_checkpoint(checkpoint, li + 1, c, n, chi, hist, settings)
    return c.detach(), n.detach(), hist

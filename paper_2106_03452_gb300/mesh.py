"""Mesh extraction on the indicator grid and the surrogate gradient of the
optimisation setting (Sec. 3.2, Eq. 6), over libdpsr's kernels
(dpsr_mesh_extract, dpsr_mesh_surrogate_splat; include/dpsr.h).

MeshPoints is a torch.autograd.Function: its forward cuts the level set
chi = level into triangles and returns points on them with their normals
(the triangle centroids, or `samples` area-weighted random points); its
backward sends dL/dp to dL/dchi through the inverse surface normal of Eq. 6,
so that a loss on mesh points reaches the oriented point cloud through the
DPSR layer's adjoint.
"""
from __future__ import annotations

import torch

from . import libdpsr as L


def extract(chi: torch.Tensor, level: float = 0.0):
    """(tris T x 3 x 3, normals T x 3) of the set chi = level (CUDA tensors)."""
    if not chi.is_cuda:
        raise ValueError("chi must be a CUDA tensor (there is no CPU path)")
    chi = chi.contiguous().float()
    r = chi.shape[0]
    st = torch.cuda.current_stream(chi.device).cuda_stream
    count = torch.zeros(1, dtype=torch.int64, device=chi.device)
    cap = max(1024, 24 * r * r)
    for _ in range(2):
        tris = torch.empty((cap, 3, 3), device=chi.device)
        nrm = torch.empty((cap, 3), device=chi.device)
        L.dpsr_mesh_extract(chi.data_ptr(), r, level, tris.data_ptr(), nrm.data_ptr(), cap, count.data_ptr(), st)
        n = int(count.item())
        if n <= cap:
            return tris[:n], nrm[:n]
        cap = n
    raise RuntimeError("mesh extraction did not converge")


def sample(tris: torch.Tensor, normals: torch.Tensor, M: int, generator=None):
    """M area-weighted uniform points on a triangle soup, with the normal of
    the triangle each falls in."""
    a = torch.linalg.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0]).norm(dim=1)
    idx = torch.multinomial(a, M, replacement=True, generator=generator)
    u = torch.rand((M, 2), device=tris.device, generator=generator)
    flip = u.sum(1) > 1
    u[flip] = 1 - u[flip]
    t = tris[idx]
    p = t[:, 0] + u[:, :1] * (t[:, 1] - t[:, 0]) + u[:, 1:] * (t[:, 2] - t[:, 0])
    return p, normals[idx]


class MeshPoints(torch.autograd.Function):
    """(points, normals) on the level set of chi; backward: Eq. 6."""

    @staticmethod
    def forward(ctx, chi, level=0.0, samples=0, generator=None):
        tris, nrm = extract(chi.detach(), level)
        if samples:
            p, n = sample(tris, nrm, samples, generator)
        else:
            p, n = tris.mean(1), nrm
        ctx.save_for_backward(p, n)
        ctx.r = chi.shape[0]
        ctx.mark_non_differentiable(n)
        return p, n

    @staticmethod
    def backward(ctx, dp, dn):
        p, n = ctx.saved_tensors
        r = ctx.r
        dchi = torch.empty((r, r, r), device=p.device)
        st = torch.cuda.current_stream(p.device).cuda_stream
        dp = dp.contiguous()
        L.dpsr_mesh_surrogate_splat(dchi.data_ptr(), r, p.contiguous().data_ptr(), n.contiguous().data_ptr(),
                                    dp.data_ptr(), p.shape[0], False, st)
        return dchi, None, None, None

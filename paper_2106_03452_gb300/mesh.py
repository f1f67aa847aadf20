"""Mesh extraction on the indicator grid and the surrogate gradient of the
optimisation setting (Sec. 3.2, Eq. 6), over libdpsr's kernels
(dpsr_mesh_extract, dpsr_mesh_surrogate_splat; include/dpsr.h).

MeshPoints is a torch.autograd.Function: its forward cuts the level set
chi = level into triangles and returns points on them with their normals
(the triangle centroids, or `samples` points drawn by area); its
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


def sample(tris: torch.Tensor, normals: torch.Tensor, M: int, seed: int = 0):
    """M points drawn uniformly by area on a triangle soup (dpsr_mesh_sample),
    with the normal of the triangle each falls in."""
    T = tris.shape[0]
    ws = torch.empty(T + (T + 1023) // 1024 + 1, dtype=torch.float64, device=tris.device)
    p = torch.empty((M, 3), device=tris.device)
    n = torch.empty((M, 3), device=tris.device)
    st = torch.cuda.current_stream(tris.device).cuda_stream
    L.dpsr_mesh_sample(tris.contiguous().data_ptr(), normals.contiguous().data_ptr(), T, M, seed, ws.data_ptr(),
                       p.data_ptr(), n.data_ptr(), st)
    return p, n


def largest_component(chi: torch.Tensor, level: float = 0.0):
    """(tris, normals) of the mesh's largest component: the surface of the
    largest connected part of {chi < level} (dpsr_largest_region)."""
    r = chi.shape[0]
    chi = chi.contiguous().float()
    st = torch.cuda.current_stream(chi.device).cuda_stream
    labels = torch.empty((r, r, r), dtype=torch.int32, device=chi.device)
    ws = torch.empty((r, r, r), dtype=torch.int32, device=chi.device)
    best = torch.zeros(1, dtype=torch.int64, device=chi.device)
    err = torch.zeros(1, dtype=torch.int32, device=chi.device)
    L.dpsr_largest_region(chi.data_ptr(), r, level, labels.data_ptr(), ws.data_ptr(), best.data_ptr(),
                          err.data_ptr(), st)
    b, e = int(best.item()), int(err.item())
    if e:
        raise RuntimeError("component labelling ran out of its iteration bound")
    if b == 0:
        return extract(chi, level)  # nothing inside: the plain extraction (empty)
    keep = 0xFFFFFFFF - (b & 0xFFFFFFFF)
    count = torch.zeros(1, dtype=torch.int64, device=chi.device)
    cap = max(1024, 24 * r * r)
    for _ in range(2):
        tris = torch.empty((cap, 3, 3), device=chi.device)
        nrm = torch.empty((cap, 3), device=chi.device)
        L.dpsr_mesh_extract_region(chi.data_ptr(), r, level, labels.data_ptr(), keep, tris.data_ptr(),
                                   nrm.data_ptr(), cap, count.data_ptr(), st)
        n = int(count.item())
        if n <= cap:
            return tris[:n], nrm[:n]
        cap = n
    raise RuntimeError("mesh extraction did not converge")


class MeshPoints(torch.autograd.Function):
    """(points, normals) on the level set of chi; backward: Eq. 6."""

    @staticmethod
    def forward(ctx, chi, level=0.0, samples=0, seed=0):
        tris, nrm = extract(chi.detach(), level)
        if samples:
            p, n = sample(tris, nrm, samples, seed)
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

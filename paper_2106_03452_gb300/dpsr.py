"""PyTorch-facing API of libdpsr: a Plan object holding the device workspace
for one grid size, and DPSRFunction, a torch.autograd.Function whose forward
and backward are the library's hand-written kernels (Sec. 3.1 of Shape As
Points and its exact adjoint). PyTorch provides device memory and streams
only; CPU tensors are rejected.
"""
from __future__ import annotations

import torch

from . import libdpsr as L


def _dev_f32(t: torch.Tensor, name: str, shape=None) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor (libdpsr has no CPU path)")
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.contiguous()


class Plan:
    """A libdpsr plan: grid size r (power of two in [8, 512]) and Gaussian
    bandwidth sigma (Eq. 3). Owns its device workspace; keeps the context of
    its last forward pass for the backward pass. box: side lengths of a
    periodic box (voxel size L_d / r per axis; points in box coordinates),
    None for the unit cube."""

    def __init__(self, r: int, sigma: float = 2.0, device=None, n_max: int | None = None, box=None):
        self.r, self.sigma = int(r), float(sigma)
        self.box = None if box is None else tuple(float(v) for v in box)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(self.device):
            if self.box is None:
                self.handle = L.dpsr_plan_create(self.r, self.sigma)
            else:
                self.handle = L.dpsr_plan_create_box(self.r, self.sigma, self.box)
            if n_max:
                L.dpsr_plan_reserve(self.handle, int(n_max))
        self._saved = None
        self.generation = 0

    def close(self):
        if getattr(self, "handle", None):
            L.dpsr_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _bind_stream(self):
        L.dpsr_plan_set_stream(self.handle, torch.cuda.current_stream(self.device).cuda_stream)

    def forward(self, points: torch.Tensor, normals: torch.Tensor, chi_out=None) -> torch.Tensor:
        points = _dev_f32(points, "points")
        normals = _dev_f32(normals, "normals", points.shape)
        if points.dim() != 2 or points.shape[1] != 3:
            raise ValueError("points must be N x 3")
        r = self.r
        if chi_out is None:
            chi_out = torch.empty((r, r, r), device=points.device, dtype=torch.float32)
        with torch.cuda.device(self.device):
            self._bind_stream()
            L.dpsr_forward(self.handle, points.data_ptr(), normals.data_ptr(), points.shape[0],
                           chi_out.data_ptr())
        # the backward reads these buffers: keep them alive
        self._saved = (points, normals, chi_out)
        self.generation += 1
        return chi_out

    def backward(self, dchi: torch.Tensor, dpoints=None, dnormals=None):
        if self._saved is None:
            raise L.DPSRError(L.DPSR_ESTATE, "dpsr_backward")
        points = self._saved[0]
        dchi = _dev_f32(dchi, "dchi", (self.r,) * 3)
        if dpoints is None:
            dpoints = torch.empty_like(points)
        if dnormals is None:
            dnormals = torch.empty_like(points)
        with torch.cuda.device(self.device):
            self._bind_stream()
            L.dpsr_backward(self.handle, dchi.data_ptr(), dpoints.data_ptr(), dnormals.data_ptr())
        return dpoints, dnormals

    def mse_grad(self, target: torch.Tensor, dchi=None) -> torch.Tensor:
        """L_DPSR (Eq. 9) of the last forward's chi against `target`: returns
        dL/dchi = (2/n)(chi - target); the loss is read by loss()."""
        target = _dev_f32(target, "target", (self.r,) * 3)
        if dchi is None:
            dchi = torch.empty_like(target)
        with torch.cuda.device(self.device):
            self._bind_stream()
            L.dpsr_mse_grad(self.handle, target.data_ptr(), dchi.data_ptr())
        self._target = target
        return dchi

    def loss(self) -> float:
        return L.dpsr_get_loss(self.handle)

    def sync(self) -> int:
        return L.dpsr_sync(self.handle)

    def check(self) -> None:
        L.check(self.sync(), "dpsr device status")

    def scalars(self):
        """(mu, s, m/|s|) of the last forward pass (Eq. 4)."""
        return L.dpsr_get_scalars(self.handle)

    def last_launches(self) -> int:
        return L.dpsr_plan_last_launches(self.handle)


class DPSRFunction(torch.autograd.Function):
    """chi = DPSR(points, normals) with the library's adjoint as backward."""

    @staticmethod
    def forward(ctx, points, normals, plan: Plan):
        chi = plan.forward(points.detach(), normals.detach())
        ctx.plan = plan
        ctx.generation = plan.generation
        return chi

    @staticmethod
    def backward(ctx, dchi):
        if ctx.plan.generation != ctx.generation:
            raise RuntimeError("the plan ran another forward pass since this one: one pending "
                               "backward per plan (use one Plan per graph node)")
        dp, dn = ctx.plan.backward(dchi.contiguous())
        return dp, dn, None


def dpsr(points: torch.Tensor, normals: torch.Tensor, plan: Plan) -> torch.Tensor:
    return DPSRFunction.apply(points, normals, plan)


class Batch:
    """Many independent solves (mixed r, uneven N) run together: every kernel
    launches once per grid size for all instances of that size, and with
    graph=True the whole forward (+ backward) sequence is one CUDA graph
    launch. Instances bind caller-owned CUDA tensors. boxes: one periodic box
    (3 side lengths) per instance, None for the unit cube."""

    def __init__(self, rs, sigmas, n_max, device=None, boxes=None):
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.rs = [int(r) for r in rs]
        with torch.cuda.device(self.device):
            if boxes is None:
                self.handle = L.dpsr_batch_create(self.rs, [float(s) for s in sigmas], [int(n) for n in n_max])
            else:
                self.handle = L.dpsr_batch_create_box(self.rs, [float(s) for s in sigmas], boxes,
                                                      [int(n) for n in n_max])
            self.stream = torch.cuda.Stream(self.device)
        L.dpsr_batch_set_stream(self.handle, self.stream.cuda_stream)
        self._bound = [None] * len(self.rs)

    def bind(self, i, points, normals, chi, dchi=None, dpoints=None, dnormals=None):
        r = self.rs[i]
        points = _dev_f32(points, "points")
        normals = _dev_f32(normals, "normals", points.shape)
        chi = _dev_f32(chi, "chi", (r, r, r))
        ptr = lambda t: t.data_ptr() if t is not None else 0
        L.dpsr_batch_bind(self.handle, i, points.data_ptr(), normals.data_ptr(), points.shape[0],
                          chi.data_ptr(), ptr(dchi), ptr(dpoints), ptr(dnormals))
        self._bound[i] = (points, normals, chi, dchi, dpoints, dnormals)

    def run(self, with_bwd=True, graph=True):
        cur = torch.cuda.current_stream(self.device)
        self.stream.wait_stream(cur)
        if graph:
            L.dpsr_batch_graph_launch(self.handle, with_bwd)
        else:
            L.dpsr_batch_forward(self.handle)
            if with_bwd:
                L.dpsr_batch_backward(self.handle)
        cur.wait_stream(self.stream)

    def sync(self) -> int:
        return L.dpsr_batch_sync(self.handle)

    def bind_target(self, i, target):
        """Target grid of instance i for train_step (L_DPSR, Eq. 9)."""
        target = _dev_f32(target, "target", (self.rs[i],) * 3)
        L.dpsr_batch_bind_target(self.handle, i, target.data_ptr())
        self._targets = getattr(self, "_targets", {})
        self._targets[i] = target

    def train_step(self):
        """One CUDA graph: forward, L_DPSR against the bound targets (gradient
        into each bound dchi), backward."""
        cur = torch.cuda.current_stream(self.device)
        self.stream.wait_stream(cur)
        L.dpsr_batch_train_step(self.handle)
        cur.wait_stream(self.stream)

    def losses(self):
        return L.dpsr_batch_losses(self.handle, len(self.rs))

    def paths(self, r: int):
        """Plane paths (tuned on the first run) of the instances of size r."""
        return L.dpsr_batch_paths(self.handle, r)

    def launches(self, with_bwd=True) -> int:
        return L.dpsr_batch_launches(self.handle, with_bwd)

    def close(self):
        if getattr(self, "handle", None):
            L.dpsr_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""Mesh extraction and the surrogate gradient of the optimisation setting
(Sec. 3.2, Eq. 6: d p_mesh / d chi = -n_mesh).

CPU pins of the reference (oracle/mesh.py), against facts that do not come
from it: the Euler characteristic of closed surfaces (sphere 2, torus 0), every
edge shared by exactly two triangles, vertices on the surface of a signed
distance field, normals along its gradient; and, for a field of unit slope,
the exact motion of the level set under chi -> chi + eps (by -eps along its
normal), which is what Eq. 6 states, against the surrogate's dL/dchi.
GPU: the extraction kernel against the reference on solved indicator grids,
the surrogate kernel against the oracle's splat, and a mesh loss through the
DPSR adjoint against the oracle chain."""
import numpy as np
import pytest

from paper_2106_03452_gb300 import synth


def _grid(r):
    j = np.arange(r) / r
    return np.meshgrid(j, j, j, indexing="ij")


def _sphere_sdf(r, c=(0.5, 0.5, 0.5), rad=0.3):
    X, Y, Z = _grid(r)
    return np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) - rad


def _torus_sdf(r, R=0.25, a=0.1):
    X, Y, Z = _grid(r)
    q = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2) - R
    return np.sqrt(q ** 2 + (Z - 0.5) ** 2) - a


def test_reference_sphere_closed_surface():
    from oracle import mesh
    r = 32
    tris, nrm = mesh.extract(_sphere_sdf(r))
    V, E, F, E2 = mesh.topology(tris)
    assert E2 == E                       # every edge in exactly two triangles
    assert V - E + F == 2                # Euler characteristic of a sphere
    p = tris.reshape(-1, 3)
    d = np.linalg.norm(p - 0.5, axis=1)
    assert np.max(np.abs(d - 0.3)) < 0.25 / r   # linear interpolation of a smooth distance
    cen = tris.mean(1)
    radial = (cen - 0.5) / np.linalg.norm(cen - 0.5, axis=1, keepdims=True)
    assert np.min(np.sum(nrm * radial, axis=1)) > 0.9   # outward: towards increasing chi


def test_reference_torus_closed_surface():
    from oracle import mesh
    tris, _ = mesh.extract(_torus_sdf(32))
    V, E, F, E2 = mesh.topology(tris)
    assert E2 == E and V - E + F == 0    # a closed surface of genus one


def test_reference_eq6_on_unit_slope_field(oracle):
    """chi(x) = |z - 1/2| - 0.2 (two planes, |grad chi| = 1): under a uniform
    shift chi + eps the level set moves by -eps along its normal, so for
    L = mean_i n_i . p_i (p_i the triangle centroids) dL/deps = -1 exactly;
    the surrogate dL/dchi of Eq. 6 sums to the same -1 (<dL/dchi, 1>)."""
    from oracle import mesh
    r = 16
    X, Y, Z = _grid(r)
    chi = np.abs(Z - 0.5) - 0.2
    tris, nrm = mesh.extract(chi)
    assert len(tris) > 0 and np.allclose(np.abs(nrm[:, 2]), 1.0)
    L = lambda t: float(np.mean(np.sum(nrm * t.mean(1), axis=1)))
    h = 1e-4
    fd = (L(mesh.extract(chi + h)[0]) - L(mesh.extract(chi - h)[0])) / (2 * h)
    assert abs(fd + 1.0) < 1e-9
    cen = tris.mean(1)
    dldp = nrm / len(nrm)
    d = mesh.surrogate_dchi(oracle, r, cen, nrm, dldp)
    assert abs(float(np.sum(d)) + 1.0) < 1e-12


# ---------------------------------------------------------------------------
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_03452_gb300 import build
    build.build()
    return torch


def _match(a, b, tol):
    """Every row of a has a row of b within tol and vice versa."""
    from scipy.spatial import cKDTree
    da, _ = cKDTree(b).query(a)
    db, _ = cKDTree(a).query(b)
    return float(max(da.max(), db.max()))


@pytest.mark.gpu
@pytest.mark.parametrize("which", ["sphere_r32", "ellipsoids_r64"])
def test_gpu_extract_matches_reference(which):
    torch = _cuda()
    from oracle import mesh as ref
    from paper_2106_03452_gb300 import mesh
    from paper_2106_03452_gb300.dpsr import Plan
    if which == "sphere_r32":
        w = synth.workload_sphere_r32()
    else:
        rng = synth.Rng(64064)
        pts, nrm = synth.ellipsoid_cloud(rng, 20000, 3)
        w = dict(r=64, sigma=2.0, points=pts, normals=nrm)
    plan = Plan(w["r"], w["sigma"])
    chi = plan.forward(torch.from_numpy(w["points"]).cuda(), torch.from_numpy(w["normals"]).cuda())
    assert plan.sync() == 0
    tris, nrm = mesh.extract(chi)
    tris_c, nrm_c = ref.extract(chi.cpu().numpy().astype(np.float64))
    assert tris.shape[0] == len(tris_c) > 0
    t, n = tris.cpu().numpy().astype(np.float64), nrm.cpu().numpy().astype(np.float64)
    assert _match(t.mean(1), tris_c.mean(1), 1e-5) <= 1e-5
    # the same triangles with the same winding: match centroid + area vector
    area = lambda q: np.cross(q[:, 1] - q[:, 0], q[:, 2] - q[:, 0])
    sc = w["r"]  # area vectors scaled to voxel units
    assert _match(np.concatenate([t.mean(1), sc * area(t)], 1),
                  np.concatenate([tris_c.mean(1), sc * area(tris_c)], 1), 1e-5) <= 1e-5
    # the kernel's unit normals: those of its own corners (in FP64), wherever
    # the direction is well conditioned (a sliver's is not in FP32)
    av = area(t)
    a = np.linalg.norm(av, axis=1)
    big = a > 0.1 * np.median(a)
    assert np.max(np.abs(n[big] - av[big] / a[big, None])) <= 1e-5
    V, E, F, E2 = ref.topology(t)
    if which == "sphere_r32":
        assert E2 == E and V - E + F == 2   # closed, genus 0
    plan.close()


@pytest.mark.gpu
def test_gpu_surrogate_matches_oracle_splat(oracle):
    torch = _cuda()
    from oracle import mesh as ref
    from paper_2106_03452_gb300 import libdpsr as L
    r, M = 32, 5000
    rng = synth.Rng(777)
    p = rng.uniform(M, 3).astype(np.float32)
    n = rng.normal(M, 3).astype(np.float32)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    g = rng.normal(M, 3).astype(np.float32)
    P, Nn, Gt = (torch.from_numpy(x).cuda() for x in (p, n, g))
    d = torch.empty((r, r, r), device="cuda")
    L.dpsr_mesh_surrogate_splat(d.data_ptr(), r, P.data_ptr(), Nn.data_ptr(), Gt.data_ptr(), M, False,
                                torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    ref_d = ref.surrogate_dchi(oracle, r, p, n, g)
    assert np.max(np.abs(d.cpu().numpy() - ref_d)) <= 1e-5 * np.max(np.abs(ref_d))


@pytest.mark.gpu
def test_gpu_mesh_loss_through_the_adjoint(oracle):
    """L = mean_i (|p_i - c| - 0.25)^2 over the mesh's triangle centroids p_i
    (the surface pulled towards radius 0.25), back to the points and normals
    of the r = 32 sphere workload: Eq. 6, then the DPSR adjoint, against the
    oracle chain on the same indicator grid."""
    torch = _cuda()
    from oracle import mesh as ref
    from paper_2106_03452_gb300.dpsr import Plan, dpsr
    from paper_2106_03452_gb300.mesh import MeshPoints
    w = synth.workload_sphere_r32()
    r, sigma = w["r"], w["sigma"]
    P = torch.from_numpy(w["points"]).cuda().requires_grad_(True)
    Nn = torch.from_numpy(w["normals"]).cuda().requires_grad_(True)
    plan = Plan(r, sigma)
    chi = dpsr(P, Nn, plan)
    p, n = MeshPoints.apply(chi)
    c = torch.tensor([0.5, 0.5, 0.5], device="cuda")
    loss = ((p - c).norm(dim=1) - 0.25).pow(2).mean()
    loss.backward()
    # oracle chain on the same grid
    chi_np = chi.detach().cpu().numpy().astype(np.float64)
    tris, nrm = ref.extract(chi_np)
    cen = tris.mean(1)
    d = np.linalg.norm(cen - 0.5, axis=1)
    dldp = (2.0 * (d - 0.25) / len(cen))[:, None] * (cen - 0.5) / d[:, None]
    dchi = ref.surrogate_dchi(oracle, r, cen, nrm, dldp)
    dp, dn = oracle.backward(r, sigma, w["points"], w["normals"], dchi)
    rel = lambda a, b: float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
    assert rel(P.grad.cpu().numpy(), dp) <= 1e-4
    assert rel(Nn.grad.cpu().numpy(), dn) <= 1e-4
    plan.close()

"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, on the
same seeded FP32 inputs. Tolerances: chi within max|d chi| / max|chi| <= 1e-5;
dpoints and dnormals within max|d| / max|ref| <= 1e-4 per tensor."""
import numpy as np
import pytest

from paper_2106_03452_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_CHI = 1e-5
TOL_GRAD = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_03452_gb300 import build
    build.build()


# Plane paths: "pencil" = independent z and y passes, "cluster" = one
# thread-block cluster per x-plane (the smallest cluster size valid for r),
# "tuned" = whatever the autotuner picks per kernel kind.
PATHS = ["pencil", "cluster"]


def _set_path(monkeypatch, path, r):
    if path == "pencil":
        monkeypatch.setenv("DPSR_PLANE_PATH", "0")
    elif path == "cluster":
        monkeypatch.setenv("DPSR_PLANE_PATH", "4" if r == 256 else "1")
    else:
        monkeypatch.delenv("DPSR_PLANE_PATH", raising=False)


_ORACLE_CACHE = {}


def _check(oracle, r, sigma, pts, nrm, dchi, tol_chi=TOL_CHI, tol_grad=TOL_GRAD, key=None):
    from gpu_util import gpu_fwd_bwd, relmax
    g = gpu_fwd_bwd(r, sigma, pts, nrm, dchi)
    assert g["status"] == 0
    ref = _ORACLE_CACHE.get(key) if key else None
    if ref is None:
        fwd = oracle.forward(r, sigma, pts.astype(np.float64), nrm.astype(np.float64), full=True)
        bwd = None
        if dchi is not None:
            bwd = oracle.backward(r, sigma, pts.astype(np.float64), nrm.astype(np.float64),
                                  dchi.astype(np.float64), mean_term=True)
        ref = (fwd, bwd)
        if key:
            _ORACLE_CACHE[key] = ref
    chi, chip, mu, s = ref[0]
    e = relmax(g["chi"], chi)
    # chi = m / |s| (chi' - mu) with s = chi'(0) - mu: an FP32 evaluation of
    # s carries a rounding of order 2^-24 max|chi'|, which the scale amplifies
    # by max|chi'| / |s|. That ratio is about 2 for surfaces (the bound stays
    # within 1 % of tol_chi) but reaches thousands for a lone point, whose
    # dipole field vanishes at the point and is tiny at the grid origin.
    cond = np.max(np.abs(chip)) / abs(s)
    tol = tol_chi + 2.0 ** -24 * cond
    assert e <= tol, f"chi parity {e:.3e} (bound {tol:.3e}, scale condition {cond:.1f})"
    gmu, gs, galpha = g["scalars"]
    assert abs(gmu - mu) <= 1e-5 * np.max(np.abs(chip)) and abs(gs - s) <= 1e-5 * abs(s) + 1e-6 * np.max(np.abs(chip))
    if dchi is not None:
        assert g["bstatus"] == 0
        dp, dn, dm = ref[1]
        # the gradient carries the same factors 1/|s| (alpha) and 1/s^2 (s_bar),
        # so the rounding of s enters it with the same relative weight
        tol_g = tol_grad + 2.0 ** -24 * cond
        en = relmax(g["dnormals"], dn)
        assert en <= tol_g, f"dnormals parity {en:.3e} (bound {tol_g:.3e})"
        # dpoints is the sum of the part through the mean of Eq. 4 (dm) and the
        # rest (dp - dm). With a handful of points the two nearly cancel, so an
        # FP32 sum is only accurate to ~1e-6 of the larger part: the bound is
        # 1e-4 of the result plus 2e-6 of the parts (the second term matters
        # only when the cancellation exceeds 50x, i.e. for N of order 1).
        scale = max(np.max(np.abs(dm)), np.max(np.abs(dp - dm)))
        err = np.max(np.abs(g["dpoints"] - dp))
        bound = tol_g * np.max(np.abs(dp)) + 2e-6 * scale
        assert err <= bound, f"dpoints parity {err / np.max(np.abs(dp)):.3e} (bound {bound:.3e})"
    return g


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("r", [8, 16, 32, 64])
@pytest.mark.parametrize("N,sigma", [(1, 2.0), (7, 0.0), (333, 2.0), (2049, 1.5)])
def test_random_clouds(oracle, monkeypatch, path, r, N, sigma):
    _set_path(monkeypatch, path, r)
    rng = synth.Rng(1000 * r + N)
    pts = (rng.uniform(N, 3) * 1.4 - 0.2).astype(np.float32)   # wraps around the unit cube
    nrm = rng.normal(N, 3).astype(np.float32)
    dchi = rng.normal(r, r, r).astype(np.float32)
    _check(oracle, r, sigma, pts, nrm, dchi)


@pytest.mark.parametrize("path", PATHS)
def test_points_on_vertices_and_faces(oracle, monkeypatch, path):
    r = 32
    _set_path(monkeypatch, path, r)
    rng = synth.Rng(4)
    N = 500
    pts = rng.uniform(N, 3)
    pts[:100] = np.floor(pts[:100] * r) / r            # exactly on vertices
    pts[100:200, 0] = np.floor(pts[100:200, 0] * r) / r  # on x faces
    pts[200:210] = 0.0
    pts[210:220] = np.float32(1.0) - np.float32(2 ** -24)  # just below 1
    pts[220:230] = -np.float32(2 ** -20)                 # just below 0
    nrm = rng.normal(N, 3)
    nrm[300:350] = 0.0                                   # muted points (zero normals)
    dchi = rng.normal(r, r, r)
    _check(oracle, r, 2.0, pts.astype(np.float32), nrm.astype(np.float32), dchi.astype(np.float32))


def test_sphere_r32(oracle):
    w = synth.workload_sphere_r32()
    _check(oracle, w["r"], w["sigma"], w["points"], w["normals"], w["dchi"])


@pytest.mark.parametrize("path", PATHS + ["tuned"])
def test_ellipsoids_r128(oracle, monkeypatch, path):
    w = synth.workload_ellipsoids_r128()
    _set_path(monkeypatch, path, w["r"])
    _check(oracle, w["r"], w["sigma"], w["points"], w["normals"], w["dchi"], key="ellipsoids_r128")


def test_ellipsoids_r128_mixed_paths(oracle, monkeypatch):
    # one path per plane kind, pinned for this grid size only: pencil forward,
    # clusters of 2, 1 and 4 for the inverse, backward and adjoint
    from paper_2106_03452_gb300 import libdpsr as L
    from gpu_util import gpu_fwd_bwd, relmax
    w = synth.workload_ellipsoids_r128()
    monkeypatch.delenv("DPSR_PLANE_PATH", raising=False)
    monkeypatch.setenv("DPSR_PLANE_PATHS_128", "0,2,1,4")
    _check(oracle, w["r"], w["sigma"], w["points"], w["normals"], w["dchi"], key="ellipsoids_r128")
    g = gpu_fwd_bwd(w["r"], w["sigma"], w["points"], w["normals"], w["dchi"])
    assert g["status"] == 0 and g["bstatus"] == 0
    assert L.dpsr_plan_clusters(g["plan"].handle) == [0, 2, 1, 4]


@pytest.mark.parametrize("r", [64, 128])
def test_split_adjoint(oracle, monkeypatch, r):
    """The adjoint plane kind as one CTA per plane and channel (path 3): the
    oracle's gradients, and the same bits as the one-CTA adjoint kernel (the
    same transforms; the channel sums in the same order)."""
    from paper_2106_03452_gb300 import libdpsr as L
    from gpu_util import gpu_fwd_bwd
    if r == 128:
        w = synth.workload_ellipsoids_r128()
        pts, nrm, dchi, sigma, key = w["points"], w["normals"], w["dchi"], w["sigma"], "ellipsoids_r128"
    else:
        rng = synth.Rng(6403)
        pts = (rng.uniform(5000, 3) * 1.4 - 0.2).astype(np.float32)   # wrapping the cube
        nrm = rng.normal(5000, 3).astype(np.float32)
        dchi = rng.normal(r, r, r).astype(np.float32)
        sigma, key = 1.5, None
    monkeypatch.delenv("DPSR_PLANE_PATH", raising=False)
    env = f"DPSR_PLANE_PATHS_{r}"
    monkeypatch.setenv(env, "1,1,1,3")
    _check(oracle, r, sigma, pts, nrm, dchi, key=key)
    # one forward, then the backward on each adjoint path: the adjoint
    # kinds see the same inputs and agree to rounding (the backward's other
    # kernels reduce with atomics, whose order can differ between runs)
    import torch
    from gpu_util import relmax
    from paper_2106_03452_gb300.dpsr import Plan
    plan = Plan(r, sigma)
    plan.forward(torch.from_numpy(pts).cuda(), torch.from_numpy(nrm).cuda())
    assert plan.sync() == 0
    G = torch.from_numpy(dchi).cuda()
    out = {}
    for paths in ("1,1,1,3", "1,1,1,1"):
        monkeypatch.setenv(env, paths)
        dp, dn = plan.backward(G)
        assert plan.sync() == 0
        out[paths] = (dp.cpu().numpy(), dn.cpu().numpy(), L.dpsr_plan_clusters(plan.handle))
    (dp3, dn3, c3), (dp1, dn1, c1) = out["1,1,1,3"], out["1,1,1,1"]
    assert c3 == [1, 1, 1, 3] and c1 == [1, 1, 1, 1]
    assert relmax(dn3, dn1) <= 1e-6 and relmax(dp3, dp1) <= 1e-6, (relmax(dn3, dn1), relmax(dp3, dp1))
    plan.close()


@pytest.mark.parametrize("path", PATHS + ["tuned"])
def test_torus_r256(oracle, monkeypatch, path):
    w = synth.workload_torus_r256()
    _set_path(monkeypatch, path, w["r"])
    dchi = synth.upstream_grad(synth.Rng(77), 256)
    _check(oracle, w["r"], w["sigma"], w["points"], w["normals"], dchi, key="torus_r256")


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("N,sigma", [(1, 2.0), (2049, 0.0)])
def test_random_clouds_r256(oracle, monkeypatch, path, N, sigma):
    """r = 256 on a lone point (nearly every plane empty) and on a sparse
    cloud with no smoothing, wrapping around the cube."""
    _set_path(monkeypatch, path, 256)
    rng = synth.Rng(256000 + N)
    pts = (rng.uniform(N, 3) * 1.4 - 0.2).astype(np.float32)
    nrm = rng.normal(N, 3).astype(np.float32)
    dchi = rng.normal(256, 256, 256).astype(np.float32)
    _check(oracle, 256, sigma, pts, nrm, dchi)


@pytest.mark.parametrize("path", ["tuned"])
def test_sphere_r512(oracle, monkeypatch, path):
    """The largest grid size, r = 512 (pencil passes only; TMA boxes split in
    two along each 512-long axis; 16384 point bins): a sphere of 20000
    points and a random upstream gradient against the FP64 oracle."""
    _set_path(monkeypatch, path, 512)
    rng = synth.Rng(5120)
    pts, nrm = synth.sphere_cloud(rng, 20000)
    dchi = rng.normal(512, 512, 512).astype(np.float32)
    g = _check(oracle, 512, 2.0, pts, nrm, dchi)
    from paper_2106_03452_gb300 import libdpsr as L
    assert L.dpsr_plan_clusters(g["plan"].handle) == [0, 0, 0, 0]


def test_degenerate_and_errors():
    import torch
    from paper_2106_03452_gb300 import libdpsr as L
    from paper_2106_03452_gb300.dpsr import Plan
    plan = Plan(32, 2.0)
    with pytest.raises(L.DPSRError) as e:
        plan.backward(torch.zeros(32, 32, 32, device="cuda"))
    assert e.value.code == L.DPSR_ESTATE
    P = torch.full((16, 3), 0.5, device="cuda")
    chi = plan.forward(P, torch.zeros(16, 3, device="cuda"))
    assert plan.sync() == L.DPSR_EDEGENERATE          # chi' = 0: no scale
    P[3, 1] = float("nan")
    plan.forward(P, torch.ones(16, 3, device="cuda"))
    assert plan.sync() == L.DPSR_EDEGENERATE          # non-finite input
    P[3, 1] = 0.25
    plan.forward(P + torch.rand_like(P) * 0.1, torch.randn(16, 3, device="cuda"))
    assert plan.sync() == L.DPSR_OK                   # status cleared, plan usable


def test_autograd_function_and_host_api(oracle):
    import torch
    from paper_2106_03452_gb300 import libdpsr as L
    from paper_2106_03452_gb300.dpsr import Plan, dpsr
    w = synth.workload_sphere_r32(N=1500)
    r = w["r"]
    plan = Plan(r, w["sigma"])
    P = torch.from_numpy(w["points"]).cuda().requires_grad_(True)
    Nn = torch.from_numpy(w["normals"]).cuda().requires_grad_(True)
    G = torch.from_numpy(w["dchi"]).cuda()
    chi = dpsr(P, Nn, plan)
    (chi * G).sum().backward()
    dp, dn = oracle.backward(r, w["sigma"], w["points"], w["normals"], w["dchi"])
    from gpu_util import relmax
    assert relmax(P.grad.cpu().numpy(), dp) <= TOL_GRAD
    assert relmax(Nn.grad.cpu().numpy(), dn) <= TOL_GRAD
    # host-buffer entry points give the same numbers as the device ones
    hp = np.ascontiguousarray(w["points"])
    hn = np.ascontiguousarray(w["normals"])
    hchi = np.zeros((r, r, r), np.float32)
    L.dpsr_forward_host(plan.handle, hp.ctypes.data, hn.ctypes.data, hp.shape[0], hchi.ctypes.data)
    assert relmax(hchi, chi.detach().cpu().numpy()) <= 1e-6
    hg = np.ascontiguousarray(w["dchi"])
    hdp = np.zeros_like(hp)
    hdn = np.zeros_like(hn)
    L.dpsr_backward_host(plan.handle, hg.ctypes.data, hdp.ctypes.data, hdn.ctypes.data)
    assert relmax(hdp, P.grad.cpu().numpy()) <= 1e-5 and relmax(hdn, Nn.grad.cpu().numpy()) <= 1e-5
    # the one-call host solve (copies overlapped on a second stream), with
    # pageable and with page-locked buffers, twice in a row
    for pinned in (False, True):
        for _ in range(2):
            bufs = [torch.from_numpy(x.copy()) for x in (hp, hn, hg)] + \
                   [torch.zeros((r, r, r)), torch.zeros(hp.shape), torch.zeros(hn.shape)]
            if pinned:
                bufs = [b.pin_memory() for b in bufs]
            tp, tn, tg, tchi, tdp, tdn = bufs
            L.dpsr_solve_host(plan.handle, tp.data_ptr(), tn.data_ptr(), hp.shape[0], tg.data_ptr(),
                              tchi.data_ptr(), tdp.data_ptr(), tdn.data_ptr())
            assert relmax(tchi.numpy(), chi.detach().cpu().numpy()) <= 1e-6
            assert relmax(tdp.numpy(), P.grad.cpu().numpy()) <= 1e-5
            assert relmax(tdn.numpy(), Nn.grad.cpu().numpy()) <= 1e-5

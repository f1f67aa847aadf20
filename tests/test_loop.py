"""The differentiable loop of the r = 256 workload: L = mean_k chi(q_k)^2 at
clean target points, gradients through the DPSR adjoint.

CPU: central finite differences of the FP64 oracle loss chain (forward,
lookup, rasterized dL/dchi, backward) at a small grid.
GPU: the step-0 gradient of the full workload (N = 100000, M = 200000,
r = 256) against the oracle chain, then 50 Adam steps that lower the loss."""
import numpy as np
import pytest

from paper_2106_03452_gb300 import synth


def _oracle_loss_grad(oracle, r, sigma, pts, nrm, q):
    chi = oracle.forward(r, sigma, pts, nrm)
    v = oracle.gather(chi, q)
    loss = float(np.mean(v * v))
    dchi = oracle.splat(r, q, (2.0 * v / len(v))[:, None])
    dp, dn = oracle.backward(r, sigma, pts, nrm, dchi)
    return loss, dp, dn


def test_loss_chain_finite_differences(oracle):
    r, sigma = 16, 2.0
    rng = synth.Rng(123)
    prims = [synth.Torus()]
    pts, nrm = synth.union_cloud(rng, prims, 400, 0.003)
    q, _ = synth.union_cloud(rng, prims, 700, 0.0)
    pts, nrm, q = pts.astype(np.float64), nrm.astype(np.float64), q.astype(np.float64)
    f = pts * r - np.floor(pts * r)  # keep coordinates away from cell faces
    pts = (np.floor(pts * r) + np.clip(f, 0.02, 0.98)) / r
    L0, dp, dn = _oracle_loss_grad(oracle, r, sigma, pts, nrm, q)
    h = 1e-6
    for (i, d) in [(0, 0), (17, 1), (230, 2), (399, 0)]:
        for arr, g in ((pts, dp), (nrm, dn)):
            a, b = arr.copy(), arr.copy()
            a[i, d] += h
            b[i, d] -= h
            la = _oracle_loss_grad(oracle, r, sigma, a if arr is pts else pts, a if arr is nrm else nrm, q)[0]
            lb = _oracle_loss_grad(oracle, r, sigma, b if arr is pts else pts, b if arr is nrm else nrm, q)[0]
            fd = (la - lb) / (2 * h)
            assert abs(fd - g[i, d]) <= 1e-6 * np.max(np.abs(g)) + 1e-12, (i, d, fd, g[i, d])


@pytest.mark.slow
def test_r256_workload_finite_differences(oracle):
    """Step 0 of the r = 256 workload itself (N = 100 000 sources, M = 200 000
    targets, sigma = 2): central finite differences of the FP64 oracle loss
    chain against its adjoint, on the entries with the largest gradients among
    points at least 2 % of a voxel away from every cell face."""
    w = synth.workload_torus_r256()
    r, sigma = w["r"], w["sigma"]
    pts, nrm, q = (w[k].astype(np.float64) for k in ("points", "normals", "targets"))
    L0, dp, dn = _oracle_loss_grad(oracle, r, sigma, pts, nrm, q)
    f = pts * r - np.floor(pts * r)
    off_faces = np.all((f > 0.02) & (f < 0.98), axis=1)
    picks = []
    for g in (dp, dn):
        mag = np.where(off_faces[:, None], np.abs(g), 0.0)
        flat = np.argsort(mag.ravel())[::-1][:3]
        picks.append([divmod(int(k), 3) for k in flat])
    h = 1e-6
    for (arr, g, sel) in ((pts, dp, picks[0]), (nrm, dn, picks[1])):
        for (i, d) in sel:
            a, b = arr.copy(), arr.copy()
            a[i, d] += h
            b[i, d] -= h
            la = _oracle_loss_grad(oracle, r, sigma, a if arr is pts else pts, a if arr is nrm else nrm, q)[0]
            lb = _oracle_loss_grad(oracle, r, sigma, b if arr is pts else pts, b if arr is nrm else nrm, q)[0]
            fd = (la - lb) / (2 * h)
            assert abs(fd - g[i, d]) <= 1e-5 * abs(g[i, d]) + 1e-9 * np.max(np.abs(g)), (i, d, fd, g[i, d])


@pytest.mark.gpu
def test_r256_loop_gradient_and_descent(oracle):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_03452_gb300 import build
    build.build()
    from paper_2106_03452_gb300.dpsr import Plan, dpsr
    from paper_2106_03452_gb300.loop import optimize, surface_loss
    w = synth.workload_torus_r256()
    r, sigma = w["r"], w["sigma"]
    P = torch.from_numpy(w["points"]).cuda().requires_grad_(True)
    Nn = torch.from_numpy(w["normals"]).cuda().requires_grad_(True)
    Q = torch.from_numpy(w["targets"]).cuda()
    plan = Plan(r, sigma, n_max=P.shape[0])
    loss = surface_loss(dpsr(P, Nn, plan), Q)
    loss.backward()
    L0, dp, dn = _oracle_loss_grad(oracle, r, sigma, w["points"], w["normals"], w["targets"])
    assert abs(float(loss.detach()) - L0) <= 1e-4 * L0
    rel = lambda a, b: float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
    assert rel(P.grad.cpu().numpy(), dp) <= 1e-4
    assert rel(Nn.grad.cpu().numpy(), dn) <= 1e-4
    hist, c, n, dt = optimize(P.detach(), Nn.detach(), Q, r=r, sigma=sigma, steps=50, plan=plan)
    assert np.isfinite(hist).all()
    assert hist[-1] < hist[0], hist[::10]
    print("loop losses", hist[::10], "s/step", dt)

"""The L_DPSR training slice of the learning setting (Sec. 3.3, Eq. 9;
supplementary Sec. B): the indicator grid of a predicted oriented cloud is
compared with a ground-truth grid (the solve of a dense sampling of the true
surface: 100 000 points at 128^3 in the paper) by the mean squared error, and
its gradient flows back to the predicted points and normals.

CPU: central finite differences of the FP64 oracle chain (forward, MSE
gradient 2 (chi - target) / n, backward) at a small grid.
GPU: the fused loss-and-gradient kernel and the batched training step (one
CUDA graph: forward, loss, backward) against that oracle chain, at r = 32
(plan) and at the paper's 128^3 with 100 000-point ground truths (batch)."""
import numpy as np
import pytest

from paper_2106_03452_gb300 import synth


def _oracle_chain(oracle, r, sigma, pts, nrm, target):
    chi = oracle.forward(r, sigma, pts, nrm)
    d = chi - target
    loss = float(np.mean(d * d))
    dchi = 2.0 * d / d.size
    dp, dn = oracle.backward(r, sigma, pts, nrm, dchi)
    return loss, dchi, dp, dn


def _pred_and_gt(seed, N_pred, N_gt, pred_sphere=True):
    """A prediction (a sphere cloud) and a ground truth (a dense sampling of a
    union of ellipsoids, no jitter): different shapes, so chi - target is of
    the order of chi itself."""
    rng = synth.Rng(seed)
    gp, gn = synth.ellipsoid_cloud(rng, N_gt, 3, jitter=0.0)
    if pred_sphere:
        pp, pn = synth.sphere_cloud(rng, N_pred, radius=0.25, jitter=0.01)
    else:
        pp, pn = synth.ellipsoid_cloud(rng, N_pred, 2, jitter=0.01)
    return pp, pn, gp, gn


def test_mse_chain_finite_differences(oracle):
    r, sigma = 16, 2.0
    pp, pn, gp, gn = _pred_and_gt(41, 300, 2000)
    pp, pn = pp.astype(np.float64), pn.astype(np.float64)
    f = pp * r - np.floor(pp * r)  # keep coordinates away from cell faces
    pp = (np.floor(pp * r) + np.clip(f, 0.02, 0.98)) / r
    target = oracle.forward(r, sigma, gp, gn)
    L0, _, dp, dn = _oracle_chain(oracle, r, sigma, pp, pn, target)
    h = 1e-6
    for (i, d) in [(0, 0), (31, 1), (150, 2), (299, 0)]:
        for arr, g in ((pp, dp), (pn, dn)):
            a, b = arr.copy(), arr.copy()
            a[i, d] += h
            b[i, d] -= h
            pa = (a, pn) if arr is pp else (pp, a)
            pb = (b, pn) if arr is pp else (pp, b)
            fd = (_oracle_chain(oracle, r, sigma, *pa, target)[0] -
                  _oracle_chain(oracle, r, sigma, *pb, target)[0]) / (2 * h)
            assert abs(fd - g[i, d]) <= 1e-6 * np.max(np.abs(g)) + 1e-12, (i, d, fd, g[i, d])


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_03452_gb300 import build
    build.build()
    return torch


@pytest.mark.gpu
def test_plan_mse_grad_matches_oracle_chain(oracle):
    torch = _cuda()
    from paper_2106_03452_gb300.dpsr import Plan
    r, sigma = 32, 2.0
    pp, pn, gp, gn = _pred_and_gt(42, 3000, 20000)
    plan = Plan(r, sigma)
    gt = plan.forward(torch.from_numpy(gp).cuda(), torch.from_numpy(gn).cuda()).clone()
    assert plan.sync() == 0
    P, Nn = torch.from_numpy(pp).cuda(), torch.from_numpy(pn).cuda()
    chi = plan.forward(P, Nn)
    dchi = plan.mse_grad(gt)
    dp, dn = plan.backward(dchi)
    assert plan.sync() == 0
    loss = plan.loss()
    target = oracle.forward(r, sigma, gp, gn)
    L0, dchi0, dp0, dn0 = _oracle_chain(oracle, r, sigma, pp, pn, target)
    assert abs(loss - L0) <= 1e-5 * L0
    assert _rel(dchi.cpu(), dchi0) <= 1e-5
    assert _rel(dp.cpu(), dp0) <= 1e-4 and _rel(dn.cpu(), dn0) <= 1e-4
    # the kernel's own arithmetic: exactly 2/n (chi - target) of its inputs
    ref = (chi.double() - gt.double()) * (2.0 / r ** 3)
    assert torch.max(torch.abs(dchi.double() - ref)).item() <= 1e-6 * torch.max(torch.abs(ref)).item()
    plan.close()


@pytest.mark.gpu
def test_batch_train_step_at_128_matches_oracle_chain(oracle):
    """Ground truths from 100 000-point samplings solved at 128^3 by a batch
    forward pass; predictions of 3000 x 7 = 21 000 points (the learning
    setting's input size times its offsets per point); one training step as a
    CUDA graph, replayed twice; two instances checked against the oracle."""
    torch = _cuda()
    from paper_2106_03452_gb300.dpsr import Batch
    r, sigma, count = 128, 2.0, 4
    data = [_pred_and_gt(500 + i, 21000, 100000, pred_sphere=(i % 2 == 0)) for i in range(count)]
    gtb = Batch([r] * count, [sigma] * count, [100000] * count)
    gts = []
    for i, (_, _, gp, gn) in enumerate(data):
        g = torch.empty((r, r, r), device="cuda")
        gtb.bind(i, torch.from_numpy(gp).cuda(), torch.from_numpy(gn).cuda(), g)
        gts.append(g)
    gtb.run(with_bwd=False, graph=False)
    assert gtb.sync() == 0
    b = Batch([r] * count, [sigma] * count, [21000] * count)
    T = []
    for i, (pp, pn, _, _) in enumerate(data):
        P, Nn = torch.from_numpy(pp).cuda(), torch.from_numpy(pn).cuda()
        chi, dchi = torch.empty((r, r, r), device="cuda"), torch.empty((r, r, r), device="cuda")
        dp, dn = torch.empty_like(P), torch.empty_like(P)
        b.bind(i, P, Nn, chi, dchi, dp, dn)
        b.bind_target(i, gts[i])
        T.append((chi, dchi, dp, dn))
    ref = {}
    for i in (0, 1):
        pp, pn, gp, gn = data[i]
        ref[i] = _oracle_chain(oracle, r, sigma, pp, pn, oracle.forward(r, sigma, gp, gn))
    for rep in range(2):  # graph capture, then replay
        for (_, dchi, dp, dn) in T:
            dchi.fill_(float("nan")); dp.fill_(float("nan")); dn.fill_(float("nan"))
        b.train_step()
        assert b.sync() == 0
        losses = b.losses()
        assert all(np.isfinite(losses))
        for i in (0, 1):
            L0, dchi0, dp0, dn0 = ref[i]
            assert abs(losses[i] - L0) <= 1e-5 * L0, (i, losses[i], L0)
            assert _rel(T[i][1].cpu(), dchi0) <= 1e-5, i
            assert _rel(T[i][2].cpu(), dp0) <= 1e-4 and _rel(T[i][3].cpu(), dn0) <= 1e-4, i
    b.close()
    gtb.close()

"""Batched solves (32 clouds, r in {64, 128}, N log-uniform in [1000, 50000]):
every instance of the batch equals its solo solve, with and without the CUDA
graph, and a sample of instances matches the FP64 oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_03452_gb300 import build
    build.build()


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("path", ["pencil", "tuned", "split"])
def test_batch_equals_solo_and_oracle(oracle, monkeypatch, path):
    import torch
    if path == "pencil":
        monkeypatch.setenv("DPSR_PLANE_PATH", "0")
    else:
        monkeypatch.delenv("DPSR_PLANE_PATH", raising=False)
    if path == "split":  # the adjoint kind as one CTA per plane and channel, batch and solo
        monkeypatch.setenv("DPSR_PLANE_PATHS_64", "1,1,1,3")
        monkeypatch.setenv("DPSR_PLANE_PATHS_128", "1,1,1,3")
    from paper_2106_03452_gb300 import synth
    from paper_2106_03452_gb300.dpsr import Batch, Plan
    inst = synth.workload_batch(count=32)
    rs = [w["r"] for w in inst]
    assert set(rs) == {64, 128}
    batch = Batch(rs, [w["sigma"] for w in inst], [w["points"].shape[0] for w in inst])
    T = []
    for i, w in enumerate(inst):
        r = w["r"]
        P = torch.from_numpy(w["points"]).cuda()
        Nn = torch.from_numpy(w["normals"]).cuda()
        G = torch.from_numpy(w["dchi"]).cuda()
        chi = torch.empty((r, r, r), device="cuda")
        dp, dn = torch.empty_like(P), torch.empty_like(P)
        batch.bind(i, P, Nn, chi, G, dp, dn)
        T.append((P, Nn, G, chi, dp, dn))
    for graph in (False, True, True):  # plain launches, graph capture, graph replay
        for (_, _, _, chi, dp, dn) in T:
            chi.fill_(float("nan")); dp.fill_(float("nan")); dn.fill_(float("nan"))
        batch.run(with_bwd=True, graph=graph)
        assert batch.sync() == 0
        for i, (P, Nn, G, chi, dp, dn) in enumerate(T):
            w = inst[i]
            plan = Plan(w["r"], w["sigma"])
            c0 = plan.forward(P, Nn).clone()
            d0, n0 = plan.backward(G)
            assert plan.sync() == 0
            assert _rel(chi.cpu(), c0.cpu()) <= 1e-5, i
            assert _rel(dp.cpu(), d0.cpu()) <= 1e-4 and _rel(dn.cpu(), n0.cpu()) <= 1e-4, i
            plan.close()
    for i in (0, 7, 31):
        w = inst[i]
        ref = oracle.forward(w["r"], w["sigma"], w["points"], w["normals"])
        assert _rel(T[i][3].cpu(), ref) <= 1e-5
        rdp, rdn = oracle.backward(w["r"], w["sigma"], w["points"], w["normals"], w["dchi"])
        assert _rel(T[i][4].cpu(), rdp) <= 1e-4 and _rel(T[i][5].cpu(), rdn) <= 1e-4
    # per grid size: bin (2), x-passes (2), combine, and one (cluster) or two
    # (pencil) launches for each of the four plane kinds
    n = batch.launches(True)
    assert 2 * 9 <= n <= 2 * 13 and (path != "pencil" or n == 2 * 13)
    if path == "split":
        assert batch.paths(64) == [1, 1, 1, 3] and batch.paths(128) == [1, 1, 1, 3]
    batch.close()


def test_batch_mixed_sigma_and_sizes(oracle):
    """One batch whose instances differ in sigma (0 = no smoothing, up to 5
    grid units: the coarse-to-fine schedule of the optimisation setting varies
    sigma per level) and in r (32 / 64): every instance matches the FP64
    oracle at its own sigma, so the per-instance Gaussian tables are not
    shared across the class."""
    import torch
    from paper_2106_03452_gb300 import synth
    from paper_2106_03452_gb300.dpsr import Batch
    sigmas = [0.0, 1.0, 2.0, 3.0, 5.0, 2.5]
    rs = [32, 64, 32, 64, 32, 64]
    inst = [synth.workload_sphere_r32(seed=200 + i, N=1500 + 300 * i) for i in range(len(rs))]
    batch = Batch(rs, sigmas, [w["points"].shape[0] for w in inst])
    T = []
    for i, w in enumerate(inst):
        r = rs[i]
        P = torch.from_numpy(w["points"]).cuda()
        Nn = torch.from_numpy(w["normals"]).cuda()
        G = torch.from_numpy(synth.upstream_grad(synth.Rng(300 + i), r)).cuda()
        chi = torch.empty((r, r, r), device="cuda")
        dp, dn = torch.empty_like(P), torch.empty_like(P)
        batch.bind(i, P, Nn, chi, G, dp, dn)
        T.append((G, chi, dp, dn))
    batch.run(with_bwd=True, graph=True)
    assert batch.sync() == 0
    for i, w in enumerate(inst):
        G, chi, dp, dn = T[i]
        ref = oracle.forward(rs[i], sigmas[i], w["points"], w["normals"])
        assert _rel(chi.cpu(), ref) <= 1e-5, (i, sigmas[i])
        rdp, rdn = oracle.backward(rs[i], sigmas[i], w["points"], w["normals"], G.cpu().numpy())
        assert _rel(dp.cpu(), rdp) <= 1e-4 and _rel(dn.cpu(), rdn) <= 1e-4, (i, sigmas[i])
    batch.close()


def test_batch_mixed_boxes_and_sigma(oracle):
    """One batch whose instances differ in their periodic box (anisotropic
    voxel sizes), in sigma and in r: every instance matches the FP64 oracle's
    box solve, so the per-instance tables and coordinate scalings are not
    shared across a class."""
    import torch
    from paper_2106_03452_gb300 import synth
    from paper_2106_03452_gb300.dpsr import Batch
    boxes = [(1.0, 0.75, 1.5), (2.0, 2.0, 0.5), (1.0, 1.0, 1.0), (0.8, 1.2, 1.0), (1.5, 1.0, 0.75)]
    sigmas = [2.0, 1.0, 2.0, 3.0, 0.0]
    rs = [32, 64, 64, 32, 64]
    inst = []
    for i, b in enumerate(boxes):
        w = synth.workload_sphere_r32(seed=400 + i, N=1500 + 400 * i)
        inst.append(((w["points"] * np.asarray(b, np.float32)).astype(np.float32), w["normals"]))
    batch = Batch(rs, sigmas, [p.shape[0] for p, _ in inst], boxes=boxes)
    T = []
    for i, (p, n) in enumerate(inst):
        r = rs[i]
        P = torch.from_numpy(p).cuda()
        Nn = torch.from_numpy(n).cuda()
        G = torch.from_numpy(synth.upstream_grad(synth.Rng(500 + i), r)).cuda()
        chi = torch.empty((r, r, r), device="cuda")
        dp, dn = torch.empty_like(P), torch.empty_like(P)
        batch.bind(i, P, Nn, chi, G, dp, dn)
        T.append((G, chi, dp, dn))
    batch.run(with_bwd=True, graph=True)
    assert batch.sync() == 0
    for i, (p, n) in enumerate(inst):
        G, chi, dp, dn = T[i]
        p64, n64 = p.astype(np.float64), n.astype(np.float64)
        ref = oracle.forward(rs[i], sigmas[i], p64, n64, box=boxes[i])
        assert _rel(chi.cpu(), ref) <= 1e-5, (i, boxes[i])
        rdp, rdn = oracle.backward(rs[i], sigmas[i], p64, n64, G.cpu().numpy().astype(np.float64), box=boxes[i])
        assert _rel(dp.cpu(), rdp) <= 1e-4 and _rel(dn.cpu(), rdn) <= 1e-4, (i, boxes[i])
    batch.close()

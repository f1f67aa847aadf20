"""The optimisation setting (Sec. 3.2; supplementary Sec. B): the Chamfer
kernel against brute force, the largest component against a graph
connected-components routine on the same adjacency, sampling on the mesh,
and a short coarse-to-fine reconstruction from a sphere."""
import numpy as np
import pytest

from paper_2106_03452_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_03452_gb300 import build
    build.build()


def test_chamfer_matches_bruteforce():
    import torch
    from paper_2106_03452_gb300.optimize import chamfer
    rng = synth.Rng(91)
    a = rng.uniform(2000, 3).astype(np.float32)
    b = rng.uniform(3000, 3).astype(np.float32)
    A = torch.from_numpy(a).cuda().requires_grad_(True)
    loss = chamfer(A, torch.from_numpy(b).cuda())
    loss.backward()
    a64, b64 = a.astype(np.float64), b.astype(np.float64)
    d = ((a64[:, None, :] - b64[None, :, :]) ** 2).sum(-1)
    iab, iba = d.argmin(1), d.argmin(0)
    ref = d.min(1).mean() + d.min(0).mean()
    assert abs(float(loss) - ref) <= 1e-6 * ref
    g = 2.0 * (a64 - b64[iab]) / len(a64)
    np.add.at(g, iba, 2.0 * (a64[iba] - b64) / len(b64))
    assert np.max(np.abs(A.grad.cpu().numpy() - g)) <= 1e-5 * np.max(np.abs(g))


def _two_spheres(r):
    j = np.arange(r) / r
    X, Y, Z = np.meshgrid(j, j, j, indexing="ij")
    big = np.sqrt((X - 0.4) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2) - 0.25
    small = np.sqrt((X - 0.82) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2) - 0.08
    return np.minimum(big, small).astype(np.float32)


def test_largest_component_and_sampling():
    import torch
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    from oracle import mesh as ref
    from paper_2106_03452_gb300 import libdpsr as L
    from paper_2106_03452_gb300.mesh import largest_component, sample
    r = 32
    chi = _two_spheres(r)
    C = torch.from_numpy(chi).cuda()
    st = torch.cuda.current_stream().cuda_stream
    labels = torch.empty((r, r, r), dtype=torch.int32, device="cuda")
    ws = torch.empty_like(labels)
    best = torch.zeros(1, dtype=torch.int64, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    L.dpsr_largest_region(C.data_ptr(), r, 0.0, labels.data_ptr(), ws.data_ptr(), best.data_ptr(), err.data_ptr(), st)
    assert int(err.item()) == 0
    lab = labels.cpu().numpy().ravel()
    # reference: components of the inside voxels joined along the seven monotone offsets
    inside = chi.ravel() < 0
    idx = np.arange(r ** 3).reshape(r, r, r)
    rows, cols = [], []
    for d in range(1, 8):
        nb = np.roll(idx, (-(d & 1), -((d >> 1) & 1), -((d >> 2) & 1)), axis=(0, 1, 2)).ravel()
        m = inside & inside[nb]
        rows.append(idx.ravel()[m])
        cols.append(nb[m])
    rows, cols = np.concatenate(rows), np.concatenate(cols)
    G = coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(r ** 3, r ** 3))
    ncomp, comp = connected_components(G, directed=False)
    sizes = np.bincount(comp[inside])
    cin = np.unique(comp[inside])
    assert len(cin) == 2
    biggest = max(cin, key=lambda c: np.sum(comp[inside] == c))
    b = int(best.item())
    assert (b >> 32) == np.sum(comp == biggest)
    keep = 0xFFFFFFFF - (b & 0xFFFFFFFF)
    assert set(np.nonzero(lab == keep)[0]) == set(np.nonzero(comp == biggest)[0])
    assert np.all((lab >= 0) == inside)
    # the largest component's mesh: the big sphere alone, closed, genus 0
    tris, nrm = largest_component(C)
    t = tris.cpu().numpy().astype(np.float64)
    V, E, F, E2 = ref.topology(t)
    assert E2 == E and V - E + F == 2
    p = t.reshape(-1, 3)
    assert np.max(np.abs(np.linalg.norm(p - [0.4, 0.5, 0.5], axis=1) - 0.25)) < 0.25 / r
    full, _ = ref.extract(chi.astype(np.float64))
    assert len(full) > len(t)  # the small sphere was dropped
    # sampling: on the triangles, reproducible, uniform by area
    P, Nn = sample(tris, nrm, 20000, seed=5)
    P2, _ = sample(tris, nrm, 20000, seed=5)
    assert torch.equal(P, P2)
    P = P.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(np.linalg.norm(P - [0.4, 0.5, 0.5], axis=1) - 0.25)) < 0.25 / r
    area = 0.5 * np.linalg.norm(np.cross(t[:, 1] - t[:, 0], t[:, 2] - t[:, 0]), axis=1)
    cen = (area[:, None] * t.mean(1)).sum(0) / area.sum()
    assert np.max(np.abs(P.mean(0) - cen)) < 3e-3
    assert np.allclose(np.linalg.norm(Nn.cpu().numpy(), axis=1), 1.0, atol=1e-5)


def test_short_reconstruction_from_a_sphere():
    """Two coarse levels (32^3 and 64^3, 150 iterations each, resampling every
    50) from a sphere towards an unoriented cloud on a torus (one connected
    object, as the resampling from the largest component assumes): the
    Chamfer distance falls well below its start and the final surface is one
    closed component."""
    import torch
    from oracle import mesh as ref
    from paper_2106_03452_gb300.mesh import largest_component
    from paper_2106_03452_gb300.dpsr import Plan
    from paper_2106_03452_gb300.optimize import reconstruct
    rng = synth.Rng(4242)
    tgt, _ = synth.union_cloud(rng, [synth.Torus()], 20000, 0.0)
    T = torch.from_numpy(tgt).cuda()
    c, n, hist = reconstruct(T, levels=((32, 2.0, 150), (64, 2.0, 150)), n_points=5000, samples=8000,
                             resample=50, seed=3)
    assert hist[-1][4] < 0.25 * hist[0][3], hist
    plan = Plan(64, 2.0)
    chi = plan.forward(c, n)
    assert plan.sync() == 0
    tris, _ = largest_component(chi)
    V, E, F, E2 = ref.topology(tris.cpu().numpy().astype(np.float64))
    assert E2 == E
    plan.close()


def test_checkpoint_and_resume(tmp_path):
    """A level-boundary checkpoint round-trips the state exactly, a resumed
    run skips the completed level (its history entry is the saved one) and
    carries on from the saved mesh, and a checkpoint of another schedule is
    refused."""
    import torch
    from paper_2106_03452_gb300.optimize import load_checkpoint, reconstruct
    rng = synth.Rng(4243)
    tgt, _ = synth.union_cloud(rng, [synth.Torus()], 10000, 0.0)
    T = torch.from_numpy(tgt).cuda()
    levels = ((32, 2.0, 60), (64, 2.0, 60))
    kw = dict(n_points=4000, samples=6000, resample=30, seed=5)
    ck = str(tmp_path / "level1.npz")
    c1, n1, h1 = reconstruct(T, levels=levels[:1], checkpoint=ck, **kw)
    # the first level alone was run with a one-level schedule: write the
    # two-level schedule's checkpoint from the same state
    lvl, c, n, chi, hist, _ = load_checkpoint(ck, T.device)
    assert lvl == 1 and torch.equal(c, c1) and torch.equal(n, n1) and hist == h1
    ck2 = str(tmp_path / "level1_of_2.npz")
    from paper_2106_03452_gb300.optimize import _settings, save_checkpoint
    save_checkpoint(ck2, 1, c, n, chi, hist, _settings(levels, kw["n_points"], kw["samples"], 2e-3, 0.7,
                                                       kw["resample"], kw["seed"]))
    c2, n2, h2 = reconstruct(T, levels=levels, resume=ck2, **kw)
    assert len(h2) == 2 and h2[0] == h1[0]          # restored, not rerun
    assert h2[1][0] == 64 and np.isfinite(h2[1][4]) and h2[1][4] < h2[1][3]
    with pytest.raises(ValueError):
        reconstruct(T, levels=levels, resume=ck, **kw)  # written with the one-level schedule

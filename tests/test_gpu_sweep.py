"""A seeded sweep over the layer's parameter space against the FP64 oracle:
grid size, point count (1 to 30 000, points wrapping the domain, some on
vertices), sigma (including 0), a periodic box or the unit cube, and the
plane path (pencil passes, one-CTA clusters, or the autotuner's choice).
Each case is drawn from the case index, so a failure names a reproducible
case. Tolerances as in the other parity tests: chi within 1e-5 of its
largest entry plus the rounding of the scale s amplified by max|chi'| / |s|,
the gradients within 1e-4 plus the same term (the mean-term cancellation of
very small N is bounded as in test_gpu_parity)."""
import numpy as np
import pytest

from paper_2106_03452_gb300 import synth

pytestmark = pytest.mark.gpu

CASES = 48


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_03452_gb300 import build
    build.build()


def _case(i):
    rng = synth.Rng(90000 + i)
    u = rng.uniform(6)
    r = [8, 16, 32, 64, 64, 128][min(int(u[0] * 6), 5)]
    N = int(round(np.exp(np.log(1.0) + (np.log(30000.0) - np.log(1.0)) * u[1])))
    sigma = 0.0 if u[2] < 0.15 else round(float(0.5 + 4.5 * u[2]), 2)
    # a box only from 50 points on: below that the two parts of dL/dpoints
    # nearly cancel, and the oracle splits them for the unit cube only
    box = None if (u[3] < 0.5 or N < 50) else tuple(float(v) for v in np.round(0.5 + 1.5 * rng.uniform(3), 3))
    path = ["pencil", "cluster", "tuned"][min(int(u[4] * 3), 2)]
    pts = rng.uniform(N, 3) * 1.3 - 0.15
    if box is None:
        k = max(1, N // 10)
        pts[:k] = np.floor(pts[:k] * r) / r             # a tenth exactly on vertices (exact in FP32)
    else:
        # box coordinates: x / L_d * r is rounded differently by the two sides,
        # so a point within rounding of a cell face may fall in different cells
        # (same chi, different one-sided gradient, reading 11): keep points
        # 1e-4 voxel off the faces
        f = pts * r - np.floor(pts * r)
        pts = (np.floor(pts * r) + np.clip(f, 1e-4, 1 - 1e-4)) / r
        pts = pts * np.asarray(box)
    nrm = rng.normal(N, 3)
    dchi = rng.normal(r, r, r)
    return r, N, sigma, box, path, pts.astype(np.float32), nrm.astype(np.float32), dchi.astype(np.float32)


@pytest.mark.parametrize("i", range(CASES))
def test_sweep(oracle, monkeypatch, i):
    from gpu_util import gpu_fwd_bwd, relmax
    from paper_2106_03452_gb300.dpsr import Plan
    r, N, sigma, box, path, pts, nrm, dchi = _case(i)
    if path == "pencil":
        monkeypatch.setenv("DPSR_PLANE_PATH", "0")
    elif path == "cluster":
        monkeypatch.setenv("DPSR_PLANE_PATH", "1")
    else:
        monkeypatch.delenv("DPSR_PLANE_PATH", raising=False)
    g = gpu_fwd_bwd(r, sigma, pts, nrm, dchi, plan=Plan(r, sigma, box=box))
    p64, n64, g64 = pts.astype(np.float64), nrm.astype(np.float64), dchi.astype(np.float64)
    try:
        chi, chip, mu, s = oracle.forward(r, sigma, p64, n64, full=True, box=box)
    except oracle.OracleError as e:     # a degenerate draw: the GPU must say so too
        assert e.code == oracle.ORACLE_EDEGENERATE and g["status"] != 0, (i, g["status"])
        return
    assert g["status"] == 0 and g["bstatus"] == 0, (i, g["status"], g.get("bstatus"))
    cond = np.max(np.abs(chip)) / abs(s)
    e = relmax(g["chi"], chi)
    assert e <= 1e-5 + 2.0 ** -24 * cond, (i, r, N, sigma, box, path, e, cond)
    dp, dn = oracle.backward(r, sigma, p64, n64, g64, box=box)
    tol_g = 1e-4 + 2.0 ** -24 * cond
    en = relmax(g["dnormals"], dn)
    assert en <= tol_g, (i, r, N, sigma, box, path, "dnormals", en)
    if box is None:
        _, _, dm = oracle.backward(r, sigma, p64, n64, g64, mean_term=True)
        scale = max(np.max(np.abs(dm)), np.max(np.abs(dp - dm)))
    else:
        scale = np.max(np.abs(dp))
    err = np.max(np.abs(g["dpoints"] - dp))
    bound = tol_g * np.max(np.abs(dp)) + (2e-6 * scale if box is None else 0.0)
    assert err <= bound, (i, r, N, sigma, box, path, "dpoints", err / np.max(np.abs(dp)))


@pytest.mark.parametrize("j", range(6))
def test_batch_sweep(j):
    """Seeded random batches (3 to 10 instances of mixed r, N, sigma and box):
    every instance equals a solo plan's solve of the same inputs, to the
    rounding of the splat's addition order (amplified, for near-degenerate
    draws, by the conditioning of the scale s)."""
    import torch
    from gpu_util import relmax
    from paper_2106_03452_gb300.dpsr import Batch, Plan
    rng = synth.Rng(70000 + j)
    count = 3 + int(rng.uniform() * 8)
    rs, sig, boxes, clouds = [], [], [], []
    for _ in range(count):
        u = rng.uniform(4)
        r = [16, 32, 64, 128][min(int(u[0] * 4), 3)]
        N = int(round(np.exp(np.log(50.0) + (np.log(20000.0) - np.log(50.0)) * u[1])))
        box = (1.0, 1.0, 1.0) if u[2] < 0.5 else tuple(float(v) for v in np.round(0.5 + 1.5 * rng.uniform(3), 3))
        pts = ((rng.uniform(N, 3) * 1.3 - 0.15) * np.asarray(box)).astype(np.float32)
        rs.append(r)
        sig.append(round(float(4.0 * u[3]), 2))
        boxes.append(box)
        clouds.append((pts, rng.normal(N, 3).astype(np.float32), rng.normal(r, r, r).astype(np.float32)))
    batch = Batch(rs, sig, [c[0].shape[0] for c in clouds], boxes=boxes)
    out = []
    for i, (p, n, g) in enumerate(clouds):
        r = rs[i]
        P, Nn, G = (torch.from_numpy(a).cuda() for a in (p, n, g))
        chi = torch.empty((r, r, r), device="cuda")
        dp, dn = torch.empty_like(P), torch.empty_like(P)
        batch.bind(i, P, Nn, chi, G, dp, dn)
        out.append((P, Nn, G, chi, dp, dn))
    batch.run(with_bwd=True, graph=True)
    assert batch.sync() == 0
    for i, (P, Nn, G, chi, dp, dn) in enumerate(out):
        plan = Plan(rs[i], sig[i], box=boxes[i])
        c0 = plan.forward(P, Nn).clone()
        d0, n0 = plan.backward(G)
        assert plan.sync() == 0
        cond = 2.0 * float(c0.abs().max())            # max|chi'| / |s| = 2 max|chi|
        tol = 1e-5 + 4 * 2.0 ** -24 * cond
        assert relmax(chi.cpu().numpy(), c0.cpu().numpy()) <= tol, (j, i, rs[i], sig[i], boxes[i])
        assert relmax(dn.cpu().numpy(), n0.cpu().numpy()) <= 10 * tol, (j, i, "dnormals")
        assert relmax(dp.cpu().numpy(), d0.cpu().numpy()) <= 10 * tol, (j, i, "dpoints")
        plan.close()
    batch.close()


@pytest.mark.parametrize("k", range(8))
def test_mesh_extraction_sweep(k):
    """Seeded random periodic fields (a few random Fourier modes, r in
    {16, 32, 64}) at random levels, a quarter of them a level equal to a
    grid value (exact ties at vertices): the kernel's triangles equal the
    numpy reference's (count, centroids and area vectors). Topology: a
    level away from every grid value gives a closed surface (every edge in
    exactly two triangles); a tie puts vertices of several edges on one grid
    point, where the tetrahedra leave a fan that is not a manifold in exact
    arithmetic too, so there the kernel's vertex, edge and face counts must
    equal the reference's. Topology is compared only where no vertex lies
    within 2e-5 voxel of a grid point without being on it: closer than that,
    FP32 coordinates (an ulp of 1.0 is 3.8e-6 voxel at r = 64) may merge a
    vertex with the grid point's, a near-tie the FP64 reference resolves."""
    import torch
    from scipy.spatial import cKDTree
    from oracle import mesh as ref
    from paper_2106_03452_gb300 import mesh
    rng = synth.Rng(74000 + k)
    u = rng.uniform(3)
    r = [16, 32, 64][min(int(u[0] * 3), 2)]
    j = np.arange(r) / r
    X, Y, Z = np.meshgrid(j, j, j, indexing="ij")
    f = np.zeros((r, r, r))
    for _ in range(5):
        m = np.floor(rng.uniform(3) * 4).astype(int)
        ph = rng.uniform(3)
        f += rng.normal() * np.cos(2 * np.pi * (m[0] * X + ph[0])) * np.cos(2 * np.pi * (m[1] * Y + ph[1])) \
            * np.cos(2 * np.pi * (m[2] * Z + ph[2]))
    chi = f.astype(np.float32)
    if u[1] < 0.25:
        level = float(chi.flat[int(u[2] * chi.size) % chi.size])   # a tie at one vertex at least
    else:
        # the midpoint of the widest gap among 64 neighbouring grid values
        srt = np.unique(chi).astype(np.float64)
        w = srt[int((0.2 + 0.6 * u[2]) * (len(srt) - 1)):][:64]
        g = int(np.argmax(np.diff(w)))
        level = float(np.float32(0.5 * (w[g] + w[g + 1])))
    tris, nrm = mesh.extract(torch.from_numpy(chi).cuda(), level)
    tris_c, _ = ref.extract(chi.astype(np.float64), level)
    assert tris.shape[0] == len(tris_c), (k, r, level)
    if len(tris_c) == 0:
        return
    t = tris.cpu().numpy().astype(np.float64)
    area = lambda q: np.cross(q[:, 1] - q[:, 0], q[:, 2] - q[:, 0])
    a = np.concatenate([t.mean(1), r * area(t)], 1)
    b = np.concatenate([tris_c.mean(1), r * area(tris_c)], 1)
    da, _ = cKDTree(b).query(a)
    db, _ = cKDTree(a).query(b)
    assert max(da.max(), db.max()) <= 1e-5, (k, r, level, da.max(), db.max())
    wr = tris_c.reshape(-1, 3) * r
    d = np.max(np.abs(wr - np.round(wr)), axis=1)  # distance of each vertex to its nearest grid point
    if np.any((d > 0) & (d < 2e-5)):
        return
    got = ref.topology(np.mod(t, 1.0))           # vertices identified across the periodic faces
    want = ref.topology(np.mod(tris_c, 1.0))
    if np.any(d == 0):
        assert got == want, (k, r, level, got, want)
    else:
        assert want[1] == want[3] and got[1] == got[3], (k, r, level, got, want)

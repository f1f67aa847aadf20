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

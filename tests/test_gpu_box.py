"""Parity of the CUDA path in a periodic box of side lengths L (voxel size
L_d / r along axis d, Eq. A1 with a per-axis voxel size) with the FP64
oracle's box solve, on the same seeded FP32 inputs, through the C ABI
(dpsr_plan_create_box). Tolerances as for the unit cube: chi within
1e-5 of max|chi| (plus the rounding of the scale s, amplified by
max|chi'| / |s|), gradients within 1e-4 of their largest entry."""
import numpy as np
import pytest

from paper_2106_03452_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_CHI = 1e-5
TOL_GRAD = 1e-4
BOXES = [(1.0, 0.75, 1.5), (2.0, 2.0, 0.5)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_03452_gb300 import build
    build.build()


def _set_path(monkeypatch, path, r):
    if path == "pencil":
        monkeypatch.setenv("DPSR_PLANE_PATH", "0")
    elif path == "cluster":
        monkeypatch.setenv("DPSR_PLANE_PATH", "4" if r == 256 else "1")
    else:
        monkeypatch.delenv("DPSR_PLANE_PATH", raising=False)


def _in_box(pts, nrm, box):
    """A unit-cube cloud stretched into the box: positions scale by L_d,
    normals (covectors) by 1 / L_d, renormalised."""
    b = np.asarray(box, np.float64)
    p = (pts.astype(np.float64) * b).astype(np.float32)
    n = nrm.astype(np.float64) / b
    n /= np.maximum(np.linalg.norm(n, axis=1, keepdims=True), 1e-30)
    return p, n.astype(np.float32)


def _check_box(oracle, r, sigma, box, pts, nrm, dchi):
    from gpu_util import gpu_fwd_bwd, relmax
    from paper_2106_03452_gb300.dpsr import Plan
    g = gpu_fwd_bwd(r, sigma, pts, nrm, dchi, plan=Plan(r, sigma, box=box))
    assert g["status"] == 0 and g["bstatus"] == 0
    p64, n64 = pts.astype(np.float64), nrm.astype(np.float64)
    chi, chip, mu, s = oracle.forward(r, sigma, p64, n64, full=True, box=box)
    dp, dn = oracle.backward(r, sigma, p64, n64, dchi.astype(np.float64), box=box)
    cond = np.max(np.abs(chip)) / abs(s)
    tol = TOL_CHI + 2.0 ** -24 * cond
    e = relmax(g["chi"], chi)
    assert e <= tol, f"chi parity {e:.3e} (bound {tol:.3e}, scale condition {cond:.1f})"
    gmu, gs, _ = g["scalars"]
    assert abs(gmu - mu) <= 1e-5 * np.max(np.abs(chip)) and abs(gs - s) <= 1e-5 * abs(s) + 1e-6 * np.max(np.abs(chip))
    tol_g = TOL_GRAD + 2.0 ** -24 * cond
    en = relmax(g["dnormals"], dn)
    assert en <= tol_g, f"dnormals parity {en:.3e} (bound {tol_g:.3e})"
    ep = relmax(g["dpoints"], dp)
    assert ep <= tol_g, f"dpoints parity {ep:.3e} (bound {tol_g:.3e})"


@pytest.mark.parametrize("path", ["pencil", "cluster"])
@pytest.mark.parametrize("box", BOXES)
@pytest.mark.parametrize("r,N,sigma", [(16, 333, 2.0), (32, 2049, 1.5), (64, 5000, 0.0)])
def test_random_clouds_in_box(oracle, monkeypatch, path, box, r, N, sigma):
    _set_path(monkeypatch, path, r)
    rng = synth.Rng(5000 + 10 * r + N)
    pts = rng.uniform(N, 3) * 1.4 - 0.2
    f = pts * r - np.floor(pts * r)                  # 1e-4 voxel off the cell faces: the
    pts = (np.floor(pts * r) + np.clip(f, 1e-4, 1 - 1e-4)) / r   # two sides round x / L differently
    pts = pts * np.asarray(box)                      # wraps around the box
    nrm = rng.normal(N, 3)
    dchi = rng.normal(r, r, r).astype(np.float32)
    _check_box(oracle, r, sigma, box, pts.astype(np.float32), nrm.astype(np.float32), dchi)


@pytest.mark.parametrize("path", ["pencil", "cluster", "tuned"])
def test_ellipsoids_in_box_r128(oracle, monkeypatch, path):
    _set_path(monkeypatch, path, 128)
    w = synth.workload_ellipsoids_r128()
    box = BOXES[0]
    pts, nrm = _in_box(w["points"], w["normals"], box)
    u = pts.astype(np.float64) / np.asarray(box) * 128
    f = u - np.floor(u)                              # 1e-4 voxel off the cell faces (see above)
    pts = ((np.floor(u) + np.clip(f, 1e-4, 1 - 1e-4)) / 128 * np.asarray(box)).astype(np.float32)
    _check_box(oracle, 128, w["sigma"], box, pts, nrm, w["dchi"])


def test_unit_box_is_the_cube(monkeypatch):
    """box = (1, 1, 1) builds the same tables and scalings as the unit-cube
    plan. The splat adds in shared memory in arrival order, so two runs agree
    to FP32 rounding, not bit for bit: both plans on the same path, within
    2e-6 of the largest entry."""
    from paper_2106_03452_gb300.dpsr import Plan
    from gpu_util import gpu_fwd_bwd, relmax
    monkeypatch.setenv("DPSR_PLANE_PATH", "0")
    w = synth.workload_sphere_r32()
    a = gpu_fwd_bwd(32, 2.0, w["points"], w["normals"], w["dchi"], plan=Plan(32, 2.0))
    b = gpu_fwd_bwd(32, 2.0, w["points"], w["normals"], w["dchi"], plan=Plan(32, 2.0, box=(1, 1, 1)))
    for k in ("chi", "dpoints", "dnormals"):
        assert relmax(b[k], a[k]) <= 2e-6, k


def test_bad_box_rejected():
    from paper_2106_03452_gb300 import libdpsr as L
    for bad in ((1.0, 0.0, 1.0), (1.0, -2.0, 1.0), (float("inf"), 1.0, 1.0), (1.0, 1.0, float("nan"))):
        with pytest.raises(L.DPSRError) as e:
            L.dpsr_plan_create_box(32, 2.0, bad)
        assert e.value.code == L.DPSR_EINVAL

"""Pins of the FP64 oracle against things other than itself: a library FFT,
dense brute force on tiny grids, closed-form Poisson solutions, exact
invariants of Eq. 4, the geometry of a sphere, and finite differences.
All CPU-only."""
import json
import math
import os

import numpy as np
import pytest

import bruteforce as bf
from paper_2106_03452_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cloud(seed, N, lo=0.0, hi=1.0):
    rng = synth.Rng(seed)
    pts = lo + (hi - lo) * rng.uniform(N, 3)
    nrm = rng.normal(N, 3)
    return pts, nrm


# --------------------------------------------------------------------------
# FFT (Eq. A3 / A4): against numpy's FFT, round trip, Parseval.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("r", [2, 4, 8, 16])
def test_fft3_matches_numpy(oracle, r):
    rng = synth.Rng(7 + r)
    g = rng.normal(r, r, r) + 1j * rng.normal(r, r, r)
    f = oracle.fft3(g)
    assert np.max(np.abs(f - np.fft.fftn(g))) <= 1e-12 * np.max(np.abs(f))
    b = oracle.fft3(g, inverse=True)
    assert np.max(np.abs(b - np.fft.ifftn(g))) <= 1e-12 * np.max(np.abs(b))
    assert np.max(np.abs(oracle.fft3(f, inverse=True) - g)) <= 1e-12 * np.max(np.abs(g))
    assert math.isclose(np.sum(np.abs(g) ** 2), np.sum(np.abs(f) ** 2) / r ** 3, rel_tol=1e-12)


# --------------------------------------------------------------------------
# Rasterization (Eq. A1-A2) against dense tent weights.
# --------------------------------------------------------------------------
def test_splat_and_gather_dense(oracle):
    r = 8
    pts, nrm = _cloud(11, 40, -0.3, 1.3)   # includes wrapped coordinates
    pts[0] = [0.0, 0.0, 0.0]               # on a vertex
    pts[1] = [0.125, 0.5, 0.999999]        # on cell faces, just below 1
    pts[2] = [-1e-9, 1.0, 2.0]
    W = bf.dense_weights(pts, r)
    V = oracle.splat(r, pts, nrm)
    ref = (W.T @ nrm).T.reshape(3, r, r, r)
    assert np.max(np.abs(V - ref)) <= 1e-12
    Wf = oracle.splat(r, pts)
    assert np.max(np.abs(Wf.ravel() - W.sum(0))) <= 1e-12
    G = synth.Rng(3).normal(r, r, r)
    assert np.max(np.abs(oracle.gather(G, pts) - W @ G.ravel())) <= 1e-12


# --------------------------------------------------------------------------
# Whole forward against direct sums (dense weights, dense DFT, Re()).
# --------------------------------------------------------------------------
@pytest.mark.parametrize("r,sigma,N", [(4, 0.0, 7), (8, 0.0, 20), (8, 1.5, 20), (8, 3.0, 13)])
def test_forward_bruteforce(oracle, r, sigma, N):
    pts, nrm = _cloud(100 + r * 10 + N, N, -0.2, 1.2)
    chi, chip, mu, s = oracle.forward(r, sigma, pts, nrm, full=True)
    bchi, bchip, bmu, bs = bf.forward(pts, nrm, r, sigma)
    sc = np.max(np.abs(bchip))
    assert np.max(np.abs(chip - bchip)) <= 1e-12 * sc
    assert abs(mu - bmu) <= 1e-12 * sc and abs(s - bs) <= 1e-12 * sc
    assert np.max(np.abs(chi - bchi)) <= 1e-11


# --------------------------------------------------------------------------
# Closed form: a plane-wave normal field sampled exactly on the vertices.
# V = nhat cos(2 pi (k.x - phi)) has divergence -2 pi |k| sin(2 pi (k.x - phi))
# (nhat = k/|k|), so the periodic Poisson solution of Eq. 1 is
# chi' = g(k) sin(2 pi (k.x - phi)) / (2 pi |k|), g(k) = exp(-2 sigma^2 |k|^2 / r^2)
# (Eq. 3). A divergence-free field (nhat orthogonal to k) gives chi' = 0.
# The cases and their amplitudes are in tests/golden/plane_waves.json.
# --------------------------------------------------------------------------
def _lattice(r):
    j = np.stack(np.meshgrid(np.arange(r), np.arange(r), np.arange(r), indexing="ij"), -1)
    return j.reshape(-1, 3) / r


def test_plane_wave_closed_form(oracle):
    with open(os.path.join(GOLDEN, "plane_waves.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        r, sigma, k, nd, phi = c["r"], c["sigma"], np.array(c["k"], float), np.array(c["n"], float), c["phi"]
        x = _lattice(r)
        wave = np.cos(2 * np.pi * (x @ k - phi))
        nrm = nd[None, :] * wave[:, None]
        if c["amplitude"] == 0.0:
            # divergence-free: chi' vanishes, so s = 0 and the layer reports a
            # degenerate scale; check through the unnormalised splat + solve
            # by adding a small reference wave along x that is not div-free.
            ref = np.array([1.0, 0, 0])[None, :] * np.cos(2 * np.pi * (x[:, 0] - 0.125))[:, None]
            _, chip_ref, _, _ = oracle.forward(r, sigma, x, ref, full=True)
            _, chip, _, _ = oracle.forward(r, sigma, x, nrm + ref, full=True)
            assert np.max(np.abs(chip - chip_ref)) <= 1e-13
            continue
        chi, chip, mu, s = oracle.forward(r, sigma, x, nrm, full=True)
        expect = c["amplitude"] * np.sin(2 * np.pi * (x @ k - phi))
        assert np.max(np.abs(chip.ravel() - expect)) <= 1e-13, c
        assert abs(mu) <= 1e-13
        assert math.isclose(s, expect[0], rel_tol=1e-10)


# --------------------------------------------------------------------------
# Exact invariants of the normalisation (Eq. 2, Eq. 4) and symmetries.
# --------------------------------------------------------------------------
def test_invariants(oracle):
    r, sigma = 16, 2.0
    rng = synth.Rng(5)
    pts = 0.2 + 0.6 * rng.uniform(300, 3)
    nrm = rng.normal(300, 3)
    chi, chip, mu, s = oracle.forward(r, sigma, pts, nrm, full=True)
    W = bf.dense_weights(pts, r)
    assert abs((W @ chi.ravel()).mean()) <= 1e-12           # chi = 0 at the points on average
    assert math.isclose(abs(chi[0, 0, 0]), 0.5, rel_tol=1e-12)
    assert np.max(np.abs(oracle.forward(r, sigma, pts, 3.7 * nrm) - chi)) <= 1e-12
    assert np.max(np.abs(oracle.forward(r, sigma, pts, -nrm) + chi)) <= 1e-12
    # chi' is linear in the normals
    n2 = rng.normal(300, 3)
    _, c1, _, _ = oracle.forward(r, sigma, pts, nrm + n2, full=True)
    _, c2, _, _ = oracle.forward(r, sigma, pts, n2, full=True)
    assert np.max(np.abs(c1 - chip - c2)) <= 1e-12 * np.max(np.abs(c1))
    # integer-voxel shift of every point circularly shifts chi'
    sh = np.array([3, -5, 7])
    _, cs, _, _ = oracle.forward(r, sigma, pts + sh / r, nrm, full=True)
    assert np.max(np.abs(cs - np.roll(chip, tuple(sh), axis=(0, 1, 2)))) <= 1e-12 * np.max(np.abs(chip))
    # swapping the x and y axes of positions and normals transposes chi'
    _, ct, _, _ = oracle.forward(r, sigma, pts[:, [1, 0, 2]], nrm[:, [1, 0, 2]], full=True)
    assert np.max(np.abs(ct - np.transpose(chip, (1, 0, 2)))) <= 1e-12 * np.max(np.abs(chip))
    # sigma = 0 is allowed (no smoothing) and differs from sigma > 0
    c0 = oracle.forward(r, 0.0, pts, nrm)
    assert np.isfinite(c0).all() and np.max(np.abs(c0 - chi)) > 1e-3


def test_degenerate_and_invalid(oracle):
    pts = np.full((4, 3), 0.5)
    with pytest.raises(oracle.OracleError) as e:
        oracle.forward(16, 2.0, pts, np.zeros((4, 3)))      # chi' = 0: s = 0
    assert e.value.code == oracle.ORACLE_EDEGENERATE
    with pytest.raises(oracle.OracleError) as e:
        oracle.forward(12, 2.0, pts, np.ones((4, 3)))       # r not a power of two
    assert e.value.code == oracle.ORACLE_EINVAL
    bad = pts.copy()
    bad[1, 2] = np.nan
    with pytest.raises(oracle.OracleError) as e:
        oracle.forward(16, 2.0, bad, np.ones((4, 3)))
    assert e.value.code == oracle.ORACLE_EDEGENERATE


# --------------------------------------------------------------------------
# Geometry: a sphere of outward normals. chi is an indicator shifted to zero
# at the points: its zero level set sits at the sphere radius, the inside is
# negative, chi(0) = +0.5 exactly (reading: positive scale, outward normals).
# --------------------------------------------------------------------------
def _trilerp(grid, p):
    r = grid.shape[0]
    x = np.asarray(p, float) * r
    i0 = np.floor(x).astype(int)
    t = x - i0
    acc = 0.0
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                w = (t[0] if dx else 1 - t[0]) * (t[1] if dy else 1 - t[1]) * (t[2] if dz else 1 - t[2])
                acc += w * grid[(i0[0] + dx) % r, (i0[1] + dy) % r, (i0[2] + dz) % r]
    return acc


def test_sphere_geometry(oracle):
    w = synth.workload_sphere_r32()
    r = w["r"]
    chi = oracle.forward(r, w["sigma"], w["points"], w["normals"])
    assert math.isclose(chi[0, 0, 0], 0.5, rel_tol=1e-12)
    c = np.array([0.5, 0.5, 0.5])
    assert chi[16, 16, 16] < -0.3                 # inside is negative
    dirs = [np.array(d, float) for d in np.ndindex(3, 3, 3) if d != (1, 1, 1)]
    for d in dirs:
        d = (d - 1) / np.linalg.norm(d - 1)
        rad = np.linspace(0.05, 0.45, 801)
        vals = np.array([_trilerp(chi, c + q * d) for q in rad])
        cross = np.nonzero((vals[:-1] < 0) & (vals[1:] >= 0))[0]
        assert len(cross) >= 1
        q0 = rad[cross[0]]
        assert abs(q0 - 0.3) <= 1.0 / r, (d, q0)


# --------------------------------------------------------------------------
# Backward: central finite differences of L = <dchi, chi> in FP64.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("r,sigma", [(8, 1.0), (16, 2.0)])
def test_backward_finite_differences(oracle, r, sigma):
    rng = synth.Rng(31 + r)
    N = 25
    pts = 0.15 + 0.7 * rng.uniform(N, 3)
    # keep every coordinate at least 1e-3 voxel away from a cell face
    f = pts * r - np.floor(pts * r)
    pts = (np.floor(pts * r) + np.clip(f, 0.01, 0.99)) / r
    nrm = rng.normal(N, 3)
    G = rng.normal(r, r, r)
    dp, dn = oracle.backward(r, sigma, pts, nrm, G)
    L = lambda p, n: float(np.sum(G * oracle.forward(r, sigma, p, n)))
    h = 1e-6
    scale_p, scale_n = np.max(np.abs(dp)), np.max(np.abs(dn))
    for (i, d) in [(0, 0), (3, 1), (7, 2), (11, 0), (24, 2)]:
        pp, pm = pts.copy(), pts.copy()
        pp[i, d] += h
        pm[i, d] -= h
        fd = (L(pp, nrm) - L(pm, nrm)) / (2 * h)
        assert abs(fd - dp[i, d]) <= 1e-6 * scale_p, (i, d, fd, dp[i, d])
        npl, nmi = nrm.copy(), nrm.copy()
        npl[i, d] += h
        nmi[i, d] -= h
        fd = (L(pts, npl) - L(pts, nmi)) / (2 * h)
        assert abs(fd - dn[i, d]) <= 1e-6 * scale_n, (i, d, fd, dn[i, d])


def test_splat_gather_adjoint(oracle):
    """<splat(c, v), G> = <v, gather(G, c)>: the rasterization of Eq. A2 and
    the trilinear lookup are transposes of each other."""
    r = 16
    rng = synth.Rng(77)
    pts = rng.uniform(50, 3) * 3 - 1
    v = rng.normal(50)
    G = rng.normal(r, r, r)
    lhs = float(np.sum(oracle.splat(r, pts, v[:, None]) * G))
    rhs = float(np.dot(v, oracle.gather(G, pts)))
    assert math.isclose(lhs, rhs, rel_tol=1e-12)


# --------------------------------------------------------------------------
# The part of dL/dpoints that flows through the mean of Eq. 4, on its own.
# Hold chi' fixed at the unperturbed points and let only mu(c) = mean_i of the
# trilinear lookup of chi' at c_i move (s = chi'(0) - mu moves with it):
#   L_mu(c) = sum_j dchi_j m / |chi'(0) - mu(c)| (chi'_j - mu(c)).
# Its central finite differences in c are the mean term the oracle returns
# separately. The rest, dL/dpoints minus that term, is the finite difference of
# L with chi' recomputed from the moved points while mu looks chi' up at the
# unmoved points (the lookup weights frozen; the change of chi' itself still
# reaches mu and s).
# --------------------------------------------------------------------------
@pytest.mark.parametrize("r,sigma,N", [(8, 1.0, 25), (16, 2.0, 3)])
def test_backward_mean_term_finite_differences(oracle, r, sigma, N):
    rng = synth.Rng(53 + r + N)
    pts = 0.15 + 0.7 * rng.uniform(N, 3)
    f = pts * r - np.floor(pts * r)
    pts = (np.floor(pts * r) + np.clip(f, 0.01, 0.99)) / r   # off the cell faces
    nrm = rng.normal(N, 3)
    G = rng.normal(r, r, r)
    dp, dn, dm = oracle.backward(r, sigma, pts, nrm, G, mean_term=True)
    _, chip, _, _ = oracle.forward(r, sigma, pts, nrm, full=True)
    m = 0.5

    def L_mu(p):
        mu = float(np.mean(oracle.gather(chip, p)))
        return float(np.sum(G * (m / abs(chip[0, 0, 0] - mu)) * (chip - mu)))

    def L_rest(p):  # the lookup weights of mu frozen at the unmoved points
        _, cp, _, _ = oracle.forward(r, sigma, p, nrm, full=True)
        mu = float(np.mean(oracle.gather(cp, pts)))
        return float(np.sum(G * (m / abs(cp[0, 0, 0] - mu)) * (cp - mu)))

    h = 1e-6
    scale = max(np.max(np.abs(dm)), np.max(np.abs(dp - dm)))
    for i in range(min(N, 6)):
        for d in range(3):
            pp, pm = pts.copy(), pts.copy()
            pp[i, d] += h
            pm[i, d] -= h
            fd = (L_mu(pp) - L_mu(pm)) / (2 * h)
            assert abs(fd - dm[i, d]) <= 1e-7 * scale, (i, d, fd, dm[i, d])
            fd = (L_rest(pp) - L_rest(pm)) / (2 * h)
            assert abs(fd - (dp[i, d] - dm[i, d])) <= 1e-7 * scale, (i, d, fd, dp[i, d] - dm[i, d])


# --------------------------------------------------------------------------
# A periodic box of side lengths L (voxel size L_d / r along axis d, Eq. A1
# with an anisotropic s). Reading: coordinates in the box, frequencies u_d =
# f_d / L_d cycles per unit length, sigma in grid units along every axis.
# --------------------------------------------------------------------------
BOX = np.array([1.0, 0.75, 1.5])


def _box_lattice(r, box):
    return _lattice(r) * box


@pytest.mark.parametrize("m,along", [((1, 2, 0), "k"), ((0, 1, 1), "k"), ((2, 0, 3), "k"),
                                     ((1, 1, 2), "perp"), ((3, 1, 0), "perp")])
def test_box_plane_wave_closed_form(oracle, m, along):
    """V = nhat cos(2 pi (k.x - phi)) on the vertices of the box lattice with
    k_d = m_d / L_d. Its divergence is -2 pi (k.nhat) sin(...), so the
    periodic solution of Eq. 1 smoothed by Eq. 3 is
    chi' = g (k.nhat) sin(2 pi (k.x - phi)) / (2 pi |k|^2), with
    g = exp(-2 sigma^2 |m|^2 / r^2). nhat = k/|k| gives the amplitude
    g / (2 pi |k|); nhat orthogonal to k gives chi' = 0 although nhat is
    not orthogonal to m."""
    r, sigma, phi = 8, 1.25, 0.15
    m = np.array(m, float)
    k = m / BOX
    if along == "k":
        nhat = k / np.linalg.norm(k)
    else:
        nhat = np.cross(k, [0.3, -0.2, 1.0])
        nhat /= np.linalg.norm(nhat)
        assert abs(nhat @ m) > 0.05
    x = _box_lattice(r, BOX)
    theta = 2 * np.pi * (x @ k - phi)
    nrm = nhat[None, :] * np.cos(theta)[:, None]
    g = math.exp(-2 * sigma ** 2 * float(m @ m) / r ** 2)
    expect = g * float(k @ nhat) * np.sin(theta) / (2 * np.pi * float(k @ k))
    ref = np.array([1.0, 0, 0])[None, :] * np.cos(2 * np.pi * (x[:, 0] - 0.125))[:, None]
    _, chip_ref, _, _ = oracle.forward(r, sigma, x, ref, full=True, box=BOX)
    _, chip, _, _ = oracle.forward(r, sigma, x, nrm + ref, full=True, box=BOX)
    assert np.max(np.abs(chip.ravel() - chip_ref.ravel() - expect)) <= 1e-13
    if along == "k":
        _, cw, mu, s = oracle.forward(r, sigma, x, nrm, full=True, box=BOX)
        assert np.max(np.abs(cw.ravel() - expect)) <= 1e-13
        assert math.isclose(s, expect[0] - mu, rel_tol=1e-10, abs_tol=1e-15)


@pytest.mark.parametrize("r,sigma,N", [(4, 0.0, 9), (8, 1.5, 20)])
def test_box_forward_bruteforce(oracle, r, sigma, N):
    pts, nrm = _cloud(900 + r + N, N, -0.2, 1.2)
    pts = pts * BOX
    chi, chip, mu, s = oracle.forward(r, sigma, pts, nrm, full=True, box=BOX)
    bchi, bchip, bmu, bs = bf.forward(pts, nrm, r, sigma, box=BOX)
    sc = np.max(np.abs(bchip))
    assert np.max(np.abs(chip - bchip)) <= 1e-12 * sc
    assert abs(mu - bmu) <= 1e-12 * sc and abs(s - bs) <= 1e-12 * sc
    assert np.max(np.abs(chi - bchi)) <= 1e-11


def test_box_cubic_scaling(oracle):
    """A cube of side L is the unit cube stretched by L: chi' and s grow by L
    (u = f / L), chi is unchanged, dL/dpoints shrinks by 1/L and dL/dnormals
    is unchanged."""
    r, sigma, L = 16, 2.0, 2.5
    rng = synth.Rng(41)
    pts = 0.2 + 0.6 * rng.uniform(60, 3)
    nrm = rng.normal(60, 3)
    G = rng.normal(r, r, r)
    chi, chip, mu, s = oracle.forward(r, sigma, pts, nrm, full=True)
    chiL, chipL, muL, sL = oracle.forward(r, sigma, L * pts, nrm, full=True, box=(L, L, L))
    assert np.max(np.abs(chiL - chi)) <= 1e-12
    assert np.max(np.abs(chipL - L * chip)) <= 1e-12 * L * np.max(np.abs(chip))
    assert math.isclose(sL, L * s, rel_tol=1e-10)
    dp, dn = oracle.backward(r, sigma, pts, nrm, G)
    dpL, dnL = oracle.backward(r, sigma, L * pts, nrm, G, box=(L, L, L))
    assert np.max(np.abs(dpL - dp / L)) <= 1e-10 * np.max(np.abs(dp))
    assert np.max(np.abs(dnL - dn)) <= 1e-10 * np.max(np.abs(dn))


def test_box_axis_permutation_and_wrap(oracle):
    """Permuting the axes of points, normals and box permutes the axes of
    chi; shifting a point by a whole box length along an axis changes
    nothing (the domain is periodic with period L_d)."""
    r, sigma = 16, 1.5
    rng = synth.Rng(43)
    pts = (0.2 + 0.6 * rng.uniform(80, 3)) * BOX
    nrm = rng.normal(80, 3)
    chi = oracle.forward(r, sigma, pts, nrm, box=BOX)
    perm = [2, 0, 1]
    chp = oracle.forward(r, sigma, pts[:, perm], nrm[:, perm], box=BOX[perm])
    assert np.max(np.abs(chp - np.transpose(chi, perm))) <= 1e-12
    sh = pts.copy()
    sh[::3] += BOX * np.array([1, -2, 3])
    assert np.max(np.abs(oracle.forward(r, sigma, sh, nrm, box=BOX) - chi)) <= 1e-12
    for bad in ([1.0, 0.0, 1.0], [1.0, -1.0, 1.0], [1.0, np.inf, 1.0], [np.nan, 1.0, 1.0]):
        with pytest.raises(oracle.OracleError) as e:
            oracle.forward(r, sigma, pts, nrm, box=bad)
        assert e.value.code == oracle.ORACLE_EINVAL


def test_box_backward_finite_differences(oracle):
    """Central differences of L = <dchi, chi> in box coordinates."""
    r, sigma, N = 8, 1.0, 20
    rng = synth.Rng(47)
    u = 0.15 + 0.7 * rng.uniform(N, 3)
    f = u * r - np.floor(u * r)
    u = (np.floor(u * r) + np.clip(f, 0.01, 0.99)) / r      # off the cell faces
    pts = u * BOX
    nrm = rng.normal(N, 3)
    G = rng.normal(r, r, r)
    dp, dn = oracle.backward(r, sigma, pts, nrm, G, box=BOX)
    L = lambda p, n: float(np.sum(G * oracle.forward(r, sigma, p, n, box=BOX)))
    h = 1e-6
    scale_p, scale_n = np.max(np.abs(dp)), np.max(np.abs(dn))
    for (i, d) in [(0, 0), (3, 1), (7, 2), (11, 1), (19, 2)]:
        pp, pm = pts.copy(), pts.copy()
        pp[i, d] += h
        pm[i, d] -= h
        fd = (L(pp, nrm) - L(pm, nrm)) / (2 * h)
        assert abs(fd - dp[i, d]) <= 1e-6 * scale_p, (i, d, fd, dp[i, d])
        npl, nmi = nrm.copy(), nrm.copy()
        npl[i, d] += h
        nmi[i, d] -= h
        fd = (L(pts, npl) - L(pts, nmi)) / (2 * h)
        assert abs(fd - dn[i, d]) <= 1e-6 * scale_n, (i, d, fd, dn[i, d])


# --------------------------------------------------------------------------
# One point on a vertex with n = e_a: V_a is a unit impulse there, so chi'
# is the circular shift of the kernel K_a = Re IDFT(H_a) (Eq. 3), written
# out here as direct sums over every frequency.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("a", [0, 1, 2])
def test_single_point_kernel(oracle, a):
    r, sigma = 8, 1.5
    j0 = np.array([3, 5, 6])
    pts = (j0 / r)[None, :]
    nrm = np.zeros((1, 3))
    nrm[0, a] = 1.0
    _, chip, _, _ = oracle.forward(r, sigma, pts, nrm, full=True)
    f = np.where(np.arange(r) < r // 2, np.arange(r), np.arange(r) - r).astype(float)
    K = np.zeros((r, r, r))
    idx = np.arange(r)
    for kx in range(r):
        for ky in range(r):
            for kz in range(r):
                k = (kx, ky, kz)
                if k == (0, 0, 0) or k[a] == r // 2:
                    continue
                u = np.array([r // 2 if k[d] == r // 2 else f[k[d]] for d in range(3)], float)
                g = math.exp(-2 * sigma ** 2 * float(u @ u) / r ** 2)
                H = g * 1j * u[a] / (-2 * math.pi * float(u @ u))
                ph = np.exp(2j * math.pi * (kx * idx[:, None, None] + ky * idx[None, :, None]
                                            + kz * idx[None, None, :]) / r)
                K += np.real(H * ph) / r ** 3
    expect = np.roll(K, tuple(j0), axis=(0, 1, 2))
    assert np.max(np.abs(chip - expect)) <= 1e-12 * np.max(np.abs(expect))


# --------------------------------------------------------------------------
# The spectral identity of Eq. 1 / Eq. 3 on the oracle's own chi': for
# k != 0 and no axis at Nyquist, -4 pi^2 |u|^2 chi~'(k) = 2 pi i g(k) u . V~(k),
# with chi~' and V~ taken by numpy's FFT of chi' and of the rasterized field.
# --------------------------------------------------------------------------
def test_spectral_identity(oracle):
    r, sigma = 16, 2.0
    pts, nrm = _cloud(61, 200, -0.1, 1.1)
    _, chip, _, _ = oracle.forward(r, sigma, pts, nrm, full=True)
    V = oracle.splat(r, pts, nrm)                       # 3 x r^3
    C = np.fft.fftn(chip)
    Vh = [np.fft.fftn(V[d]) for d in range(3)]
    f = np.fft.fftfreq(r, 1.0 / r)
    U = np.stack(np.meshgrid(f, f, f, indexing="ij"))
    u2 = (U ** 2).sum(0)
    g = np.exp(-2 * sigma ** 2 * u2 / r ** 2)
    lhs = -4 * math.pi ** 2 * u2 * C
    rhs = 2j * math.pi * g * sum(U[d] * Vh[d] for d in range(3))
    ok = (u2 > 0) & np.all(np.abs(U) < r // 2, axis=0)
    assert np.max(np.abs(lhs - rhs)[ok]) <= 1e-10 * np.max(np.abs(rhs[ok]))


# --------------------------------------------------------------------------
# The whole linearisation at once: the directional derivative of
# L = <dchi, chi> along a random direction in (points, normals), by central
# differences, equals <grad, direction> from the backward pass.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("r,sigma,N", [(8, 1.0, 30), (16, 2.0, 60)])
def test_jvp_matches_vjp(oracle, r, sigma, N):
    rng = synth.Rng(71 + r)
    u = 0.15 + 0.7 * rng.uniform(N, 3)
    f = u * r - np.floor(u * r)
    pts = (np.floor(u * r) + np.clip(f, 0.01, 0.99)) / r
    nrm = rng.normal(N, 3)
    G = rng.normal(r, r, r)
    dp, dn = oracle.backward(r, sigma, pts, nrm, G)
    Dp, Dn = rng.normal(N, 3), rng.normal(N, 3)
    h = 1e-7
    L = lambda p, n: float(np.sum(G * oracle.forward(r, sigma, p, n)))
    fd = (L(pts + h * Dp, nrm + h * Dn) - L(pts - h * Dp, nrm - h * Dn)) / (2 * h)
    an = float(np.sum(dp * Dp) + np.sum(dn * Dn))
    assert abs(fd - an) <= 1e-6 * max(abs(an), np.sum(np.abs(dp * Dp)) + np.sum(np.abs(dn * Dn)))

"""Stage-level parity: the forward pass's intermediate spectra, read back
through dpsr_debug_read_spectrum, against the same quantities computed in
FP64 from the oracle's rasterization (Eq. A1-A2) and its chi' (Eq. A8) with
numpy's FFT, so that each stage is checked on its own and a pair of errors
cannot cancel in the final chi. Both plane paths."""
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


def _fft_yz(a):
    """Unnormalised DFT over y and the z half spectrum of a [x][y][z] grid."""
    return np.fft.fft(np.fft.rfft(a, axis=2), axis=1)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("path", ["0", "1"])
@pytest.mark.parametrize("r,N", [(32, 1500), (64, 4000), (128, 20000)])
def test_forward_stages(oracle, monkeypatch, path, r, N):
    import torch
    from paper_2106_03452_gb300 import libdpsr as L
    from paper_2106_03452_gb300.dpsr import Plan
    monkeypatch.setenv("DPSR_PLANE_PATH", path)
    sigma = 2.0
    rng = synth.Rng(6100 + r)
    pts = (rng.uniform(N, 3) * 1.4 - 0.2).astype(np.float32)
    nrm = rng.normal(N, 3).astype(np.float32)
    plan = Plan(r, sigma)
    plan.forward(torch.from_numpy(pts).cuda(), torch.from_numpy(nrm).cuda())
    assert plan.sync() == 0
    got = [L.dpsr_debug_read_spectrum(plan.handle, k, r).astype(np.complex128) for k in range(4)]
    p64, n64 = pts.astype(np.float64), nrm.astype(np.float64)
    V = oracle.splat(r, p64, n64)                     # 3 x r^3: v_x, v_y, v_z
    w = oracle.splat(r, p64).reshape(r, r, r)         # the weight field
    _, chip, _, _ = oracle.forward(r, sigma, p64, n64, full=True)
    k = np.arange(r)
    uy = np.where(k < r // 2, k, k - r).astype(float)
    uy[r // 2] = 0.0                                  # Nyquist: no derivative term
    uz = np.arange(r // 2 + 1, dtype=float)
    uz[r // 2] = 0.0
    Vy, Vz = _fft_yz(V[1].reshape(r, r, r)), _fft_yz(V[2].reshape(r, r, r))
    D = 1j * uy[None, :, None] * Vy + 1j * uz[None, None, :] * Vz
    C = _fft_yz(V[0].reshape(r, r, r))
    W = _fft_yz(w)
    P = r * _fft_yz(chip)
    for name, g, e in (("D", got[0], D), ("C", got[1], C), ("W", got[2], W), ("P", got[3], P)):
        assert _rel(g, e) <= (5e-6 if name != "P" else 1e-5), (name, _rel(g, e))
    # Backward: G_bar = alpha dchi + s_bar e_0 + (mu_bar / N) w (the adjoint
    # of Eq. 4), F = G(k) FFT3(G_bar) / r^3, Q1 = r IFFT_x(F), Q2 = r IFFT_x(-i u_x F)
    with pytest.raises(L.DPSRError) as e:
        L.dpsr_debug_read_spectrum(plan.handle, 4, r)  # no backward yet
    assert e.value.code == L.DPSR_ESTATE
    dchi = rng.normal(r, r, r).astype(np.float32)
    plan.backward(torch.from_numpy(dchi).cuda())
    assert plan.sync() == 0
    with pytest.raises(L.DPSRError) as e:
        L.dpsr_debug_read_spectrum(plan.handle, 0, r)   # the backward reused the buffers
    assert e.value.code == L.DPSR_ESTATE
    q1, q2 = (L.dpsr_debug_read_spectrum(plan.handle, k, r).astype(np.complex128) for k in (4, 5))
    _, chip, mu, s_ = oracle.forward(r, sigma, p64, n64, full=True)
    g = dchi.astype(np.float64)
    alpha = 0.5 / abs(s_)
    s_bar = -0.5 * np.sign(s_) * float(np.sum(g * (chip - mu))) / s_ ** 2
    mu_bar = -alpha * float(np.sum(g)) - s_bar
    Gb = alpha * g + (mu_bar / N) * w
    Gb[0, 0, 0] += s_bar
    Gh = np.fft.fftn(np.fft.rfft(Gb, axis=2), axes=(0, 1))
    ua = np.where(k < r // 2, k, k - r).astype(float)
    ua2 = ua.copy()
    ua2[r // 2] = r // 2
    uzz = np.arange(r // 2 + 1, dtype=float)
    U2 = ua2[:, None, None] ** 2 + ua2[None, :, None] ** 2 + uzz[None, None, :] ** 2
    Gk = np.exp(-2 * sigma ** 2 * U2 / r ** 2) / (-2 * np.pi * np.where(U2 > 0, U2, 1.0))
    Gk[0, 0, 0] = 0.0
    F = Gk * Gh / r ** 3
    ux = ua.copy()
    ux[r // 2] = 0.0
    Q1 = r * np.fft.ifft(F, axis=0)
    Q2 = r * np.fft.ifft(-1j * ux[:, None, None] * F, axis=0)
    assert _rel(q1, Q1) <= 2e-5, ("Q1", _rel(q1, Q1))
    assert _rel(q2, Q2) <= 2e-5, ("Q2", _rel(q2, Q2))
    plan.close()

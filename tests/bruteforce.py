"""Brute-force restatements used to pin the oracle on tiny inputs.

These are deliberately different formulations of the same definitions:
  - trilinear weights as the tent function T(c, s*j + c0, s) of Eq. A1,
    evaluated densely over ALL vertices with the periodic minimum-image
    distance (not the 8-neighbour floor/ceil path of the oracle);
  - the 3D DFT of Eq. A3/A4 as a dense r^3 x r^3 matrix of direct sums
    (not a factorised FFT);
  - Nyquist handled by taking Re() of a full complex inverse transform with
    u_a = +r/2 (not by zeroing terms).
Only for r <= 8.
"""
import numpy as np


def dense_weights(points, r):
    """N x r^3 matrix of T(c_i, j/r, 1/r) = prod_d max(0, 1 - r*|c_d - j_d/r|_periodic)."""
    pts = np.asarray(points, np.float64).reshape(-1, 3)
    j = np.arange(r) / r
    fac = []
    for d in range(3):
        diff = pts[:, d:d + 1] - j[None, :]
        diff = diff - np.round(diff)  # minimum image on the unit torus
        fac.append(np.maximum(0.0, 1.0 - r * np.abs(diff)))
    w = fac[0][:, :, None, None] * fac[1][:, None, :, None] * fac[2][:, None, None, :]
    return w.reshape(pts.shape[0], r ** 3)


def dft_matrix(r, sign=-1):
    idx = np.stack(np.meshgrid(np.arange(r), np.arange(r), np.arange(r), indexing="ij"), -1).reshape(-1, 3)
    phase = (idx @ idx.T) % r
    return np.exp(sign * 2j * np.pi * phase / r)


def freqs_plus_nyquist(r):
    """u_a(k) = k for k <= r/2 (Nyquist taken as +r/2), k - r above."""
    k = np.arange(r)
    return np.where(k <= r // 2, k, k - r).astype(np.float64)


def forward(points, normals, r, sigma, m=0.5, box=(1.0, 1.0, 1.0)):
    """chi, chi', mu, s by direct sums (Eq. 3, Eq. 4). box: side lengths of
    the periodic domain; the grid vertex j sits at j_d L_d / r, the tent
    weight of Eq. A1 has half-width L_d / r along axis d, frequencies are
    f_d / L_d cycles per unit length and the Gaussian's sigma is in grid
    units (f_d / r)."""
    box = np.asarray(box, np.float64)
    W = dense_weights(np.asarray(points, np.float64).reshape(-1, 3) / box, r)   # tent in grid units
    V = W.T @ np.asarray(normals, np.float64).reshape(-1, 3)     # n x 3 (Eq. A2)
    E = dft_matrix(r, -1)
    Vh = E @ V                                                   # n x 3 (Eq. A3)
    u1 = freqs_plus_nyquist(r)
    F = np.stack(np.meshgrid(u1, u1, u1, indexing="ij"), -1).reshape(-1, 3)
    U = F / box
    u2 = (U ** 2).sum(1)
    g = np.exp(-2.0 * sigma ** 2 * (F ** 2).sum(1) / r ** 2)
    with np.errstate(divide="ignore", invalid="ignore"):
        chih = g * (1j * (U * Vh).sum(1)) / (-2.0 * np.pi * u2)
    chih[0] = 0.0
    chip = np.real(dft_matrix(r, +1) @ chih) / r ** 3          # Eq. A8, Re()
    mu = (W @ chip).mean()
    s = chip[0] - mu
    chi = m / abs(s) * (chip - mu)
    return chi.reshape(r, r, r), chip.reshape(r, r, r), mu, s

"""Seeded synthetic oriented point clouds for the DPSR layer.

This module holds no arithmetic of the method itself: it only draws shapes
(spheres, ellipsoid unions, a torus) and upstream gradients from a
counter-based SplitMix64 stream, so that the CUDA path and the FP64 oracle
receive the very same FP32 arrays. It imports nothing from the rest of the
package.

Workloads (all in the unit cube, the domain of the DPSR grid):
  sphere       N points on a sphere of radius 0.3 at the cube centre, outward
               unit normals, position jitter N(0, 0.005^2).
  ellipsoids   area-uniform samples of the boundary of a union of K random
               ellipsoids (semi-axes U[0.08, 0.25], centres U[0.25, 0.75]^3,
               uniform random rotations), analytic outward normals.
  torus        a torus (R = 0.25, tube 0.08, axis z, centred) united with K
               random ellipsoids.
The paper's own inputs are scanned or ShapeNet shapes (Sec. 4); these stand in
for them with the same kind of structure: points concentrated on closed
surfaces, unit normals, Gaussian position noise.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class Rng:
    """SplitMix64 (Steele, Lea, Flood 2014) as a counter-based stream:
    output i is mix(seed + (i + 1) * gamma)."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.counter = 0

    def u64(self, n: int) -> np.ndarray:
        idx = np.arange(self.counter + 1, self.counter + n + 1, dtype=np.uint64)
        self.counter += n
        z = self.seed + idx * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))

    def uniform(self, *shape) -> np.ndarray:
        n = int(np.prod(shape)) if shape else 1
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return u.reshape(shape) if shape else u[0]

    def normal(self, *shape) -> np.ndarray:
        """Box-Muller: two uniforms per normal (the sine half is discarded)."""
        n = int(np.prod(shape)) if shape else 1
        u = self.uniform(2 * n)
        u1, u2 = u[0::2], u[1::2]
        z = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)
        return z.reshape(shape) if shape else z[0]


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _rotation(rng: Rng) -> np.ndarray:
    """Uniform random rotation from a uniform unit quaternion (Shoemake)."""
    u1, u2, u3 = rng.uniform(3)
    a, b = math.sqrt(1 - u1), math.sqrt(u1)
    x, y = a * math.sin(2 * math.pi * u2), a * math.cos(2 * math.pi * u2)
    z, w = b * math.sin(2 * math.pi * u3), b * math.cos(2 * math.pi * u3)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


@dataclass
class Ellipsoid:
    centre: np.ndarray
    axes: np.ndarray
    rot: np.ndarray  # columns: the ellipsoid's local axes in world coordinates

    @staticmethod
    def random(rng: Rng, lo=0.08, hi=0.25, clo=0.25, chi=0.75) -> "Ellipsoid":
        axes = lo + (hi - lo) * rng.uniform(3)
        centre = clo + (chi - clo) * rng.uniform(3)
        return Ellipsoid(centre, axes, _rotation(rng))

    def inside(self, p):
        q = (p - self.centre) @ self.rot
        return np.sum((q / self.axes) ** 2, axis=-1) < 1.0

    def sample(self, rng: Rng, n: int):
        """Area-uniform boundary samples: a uniform sphere direction d maps to
        a * d, accepted with probability proportional to the area element."""
        a = self.axes
        jmax = 1.0 / a.min()
        pts, nrm, got = [], [], 0
        while got < n:
            m = max(64, int(2.2 * (n - got)) + 16)
            d = _unit(rng.normal(m, 3))
            jac = np.linalg.norm(d / a, axis=1)
            keep = rng.uniform(m) * jmax < jac
            d = d[keep]
            pts.append(self.centre + (a * d) @ self.rot.T)
            nrm.append(_unit((d / a) @ self.rot.T))
            got += d.shape[0]
        return np.concatenate(pts)[:n], np.concatenate(nrm)[:n]

    def area(self, rng: Rng, m: int = 8192) -> float:
        d = _unit(rng.normal(m, 3))
        return float(4 * math.pi * np.prod(self.axes) * np.mean(np.linalg.norm(d / self.axes, axis=1)))


@dataclass
class Torus:
    centre: np.ndarray = field(default_factory=lambda: np.full(3, 0.5))
    R: float = 0.25
    tube: float = 0.08

    def inside(self, p):
        q = p - self.centre
        rho = np.sqrt(q[:, 0] ** 2 + q[:, 1] ** 2)
        return (rho - self.R) ** 2 + q[:, 2] ** 2 < self.tube ** 2

    def sample(self, rng: Rng, n: int):
        pts, nrm, got = [], [], 0
        while got < n:
            m = max(64, int(1.5 * (n - got)) + 16)
            th = 2 * math.pi * rng.uniform(m)
            ph = 2 * math.pi * rng.uniform(m)
            keep = rng.uniform(m) * (self.R + self.tube) < self.R + self.tube * np.cos(ph)
            th, ph = th[keep], ph[keep]
            nn = np.stack([np.cos(ph) * np.cos(th), np.cos(ph) * np.sin(th), np.sin(ph)], 1)
            rr = self.R + self.tube * np.cos(ph)
            p = self.centre + np.stack([rr * np.cos(th), rr * np.sin(th), self.tube * np.sin(ph)], 1)
            pts.append(p)
            nrm.append(nn)
            got += p.shape[0]
        return np.concatenate(pts)[:n], np.concatenate(nrm)[:n]

    def area(self, rng: Rng, m: int = 0) -> float:
        return 4 * math.pi ** 2 * self.R * self.tube


def union_cloud(rng: Rng, prims, N: int, jitter: float):
    """N area-uniform samples of the boundary of the union of the primitives,
    with their outward normals, plus N(0, jitter^2) position noise. Points of
    one primitive lying inside another are rejected; counts are proportional
    to each primitive's visible boundary area (Monte-Carlo estimate)."""
    vis = []
    for i, p in enumerate(prims):
        x, _ = p.sample(rng, 2048)
        out = np.ones(x.shape[0], bool)
        for j, q in enumerate(prims):
            if j != i:
                out &= ~q.inside(x)
        vis.append(p.area(rng) * out.mean())
    vis = np.asarray(vis)
    if vis.sum() <= 0:
        vis = np.ones(len(prims))
    share = N * vis / vis.sum()
    counts = np.floor(share).astype(np.int64)
    rem = N - counts.sum()
    for i in np.argsort(-(share - counts), kind="stable")[:rem]:
        counts[i] += 1
    P, Nn = [], []
    for i, p in enumerate(prims):
        need = int(counts[i])
        while need > 0:
            x, nv = p.sample(rng, max(need, 64))
            ok = np.ones(x.shape[0], bool)
            for j, q in enumerate(prims):
                if j != i:
                    ok &= ~q.inside(x)
            x, nv = x[ok][:need], nv[ok][:need]
            P.append(x)
            Nn.append(nv)
            need -= x.shape[0]
    pts = np.concatenate(P)
    nrm = np.concatenate(Nn)
    pts = pts + jitter * rng.normal(*pts.shape)
    return pts.astype(np.float32), nrm.astype(np.float32)


def sphere_cloud(rng: Rng, N: int, radius=0.3, centre=(0.5, 0.5, 0.5), jitter=0.005):
    d = _unit(rng.normal(N, 3))
    pts = np.asarray(centre) + radius * d + jitter * rng.normal(N, 3)
    return pts.astype(np.float32), d.astype(np.float32)


def ellipsoid_cloud(rng: Rng, N: int, n_ellipsoids: int, jitter=0.003):
    prims = [Ellipsoid.random(rng) for _ in range(n_ellipsoids)]
    return union_cloud(rng, prims, N, jitter)


def torus_cloud(rng: Rng, N: int, n_ellipsoids: int = 2, jitter=0.003):
    prims = [Torus()] + [Ellipsoid.random(rng) for _ in range(n_ellipsoids)]
    return union_cloud(rng, prims, N, jitter)


def upstream_grad(rng: Rng, r: int) -> np.ndarray:
    """dL/dchi ~ N(0, 1) over the r^3 grid, FP32."""
    return rng.normal(r, r, r).astype(np.float32)


def log_uniform_int(rng: Rng, lo: int, hi: int) -> int:
    return int(round(math.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * rng.uniform())))


# ---------------------------------------------------------------------------
# The five workloads. Seeds are 1000 + workload index.
# ---------------------------------------------------------------------------
SIGMA = 2.0


def workload_sphere_r32(seed: int = 1000, N: int = 3000):
    """Plain fwd+bwd, r = 32: N = 3000 on a sphere (radius 0.3) + dchi."""
    rng = Rng(seed)
    pts, nrm = sphere_cloud(rng, N)
    return dict(name="sphere_r32", r=32, sigma=SIGMA, points=pts, normals=nrm,
                dchi=upstream_grad(rng, 32))


def workload_ellipsoids_r128(seed: int = 1001, N: int = 20000):
    """Plain fwd+bwd, r = 128: N = 20000 on a union of 4 ellipsoids + dchi."""
    rng = Rng(seed)
    pts, nrm = ellipsoid_cloud(rng, N, 4)
    return dict(name="ellipsoids4_r128", r=128, sigma=SIGMA, points=pts, normals=nrm,
                dchi=upstream_grad(rng, 128))


def workload_torus_r256(seed: int = 1002, N: int = 100000, M: int = 200000):
    """Differentiable loop, r = 256: N = 100000 noisy source points on a torus
    united with 2 ellipsoids, and M = 200000 clean target points on the same
    surface."""
    rng = Rng(seed)
    prims = [Torus()] + [Ellipsoid.random(rng) for _ in range(2)]
    pts, nrm = union_cloud(rng, prims, N, 0.003)
    q, _ = union_cloud(rng, prims, M, 0.0)
    return dict(name="torus_r256", r=256, sigma=SIGMA, points=pts, normals=nrm, targets=q)


def workload_batch(seed: int = 1003, count: int = 32, n_lo=1000, n_hi=50000, rs=(64, 128)):
    """Batched: `count` clouds, each a union of 1-6 ellipsoids, N log-uniform
    in [n_lo, n_hi], r uniform over `rs`, with dchi."""
    rng = Rng(seed)
    out = []
    for _ in range(count):
        k = 1 + int(rng.uniform() * 6) % 6
        N = log_uniform_int(rng, n_lo, n_hi)
        r = rs[int(rng.uniform() * len(rs)) % len(rs)]
        pts, nrm = ellipsoid_cloud(rng, N, k)
        out.append(dict(r=r, sigma=SIGMA, points=pts, normals=nrm, dchi=upstream_grad(rng, r)))
    return out


def serving_trace(seed: int = 1004, rate: float = 200.0, duration_s: float = 60.0,
                  n_lo=1000, n_hi=200000, rs=(64, 128, 256), r_probs=(0.5, 0.35, 0.15),
                  p_backward=0.3):
    """Serving: Poisson arrivals at `rate` req/s. Each request: arrival time,
    r, N, number of ellipsoids, whether it asks for the backward pass and the
    seed of its own cloud (drawn lazily with `request_inputs`)."""
    rng = Rng(seed)
    t, reqs = 0.0, []
    cdf = np.cumsum(r_probs)
    while True:
        t += -math.log1p(-rng.uniform()) / rate
        if t >= duration_s:
            break
        u = rng.uniform()
        r = rs[int(np.searchsorted(cdf, u, side="right")) if u < cdf[-1] else len(rs) - 1]
        reqs.append(dict(t=t, r=r, N=log_uniform_int(rng, n_lo, n_hi),
                         k=1 + int(rng.uniform() * 6) % 6, backward=bool(rng.uniform() < p_backward),
                         seed=int(rng.u64(1)[0])))
    return reqs


def request_inputs(req):
    rng = Rng(req["seed"])
    pts, nrm = ellipsoid_cloud(rng, req["N"], req["k"])
    dchi = upstream_grad(rng, req["r"]) if req["backward"] else None
    return pts, nrm, dchi

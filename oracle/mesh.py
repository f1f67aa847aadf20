"""CPU reference of the mesh extraction and of the surrogate gradient of the
optimisation setting (Sec. 3.2, Eq. 6). TEST INFRASTRUCTURE: only the tests
use it; it shares no code with the GPU library.

Extraction: every cube of the periodic grid is cut into the six tetrahedra
of Kuhn's triangulation (corner 000 to corner 111 along the three axes in
each of the 3! orders); inside a tetrahedron the field is taken as the
linear interpolant of its corner values, whose zero set is a triangle (one
corner of a different sign) or a quadrilateral (two and two). A vertex on
the edge from a to b sits at a + t (b - a), t = f(a) / (f(a) - f(b)), with a
the lower endpoint (the tetrahedra's edges are monotone along the axes).
Triangles are oriented so that their normal points towards increasing f.

Surrogate (Eq. 6): dL/dchi = sum_i (dL/dp_i . (-n_i)) delta(p_i), put on the
grid by the transpose of the trilinear lookup, i.e. the oracle's splat.
"""
from __future__ import annotations

import itertools

import numpy as np


def _tets():
    out = []
    for perm in itertools.permutations(range(3)):
        c = [0, 0, 0]
        path = [tuple(c)]
        for ax in perm:
            c[ax] = 1
            path.append(tuple(c))
        out.append(path)
    return out  # six lists of four corner offsets (x, y, z), monotone


TETS = _tets()


def extract(chi, level=0.0):
    """Triangles (T x 3 x 3, float64, unit-cube coordinates, unwrapped) and
    their unit normals (T x 3) of the set chi = level."""
    f = np.asarray(chi, np.float64) - level
    r = f.shape[0]
    neg = f < 0
    # cubes with corners of both signs
    corners = [np.roll(neg, (-dx, -dy, -dz), axis=(0, 1, 2)) for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)]
    anyn = np.logical_or.reduce(corners)
    alln = np.logical_and.reduce(corners)
    cells = np.argwhere(anyn & ~alln)
    tris, nrms = [], []
    for (i, j, k) in cells:
        o = np.array([i, j, k], np.float64)
        def val(c):
            return f[(i + c[0]) % r, (j + c[1]) % r, (k + c[2]) % r]
        for tet in TETS:
            v = [val(c) for c in tet]
            s = [x < 0 for x in v]
            nneg = sum(s)
            if nneg in (0, 4):
                continue
            pos = [np.array(c, np.float64) for c in tet]

            def vert(a, b):  # a < b along the tetrahedron's monotone vertex order
                if a > b:
                    a, b = b, a
                t = v[a] / (v[a] - v[b])
                return (o + pos[a] + t * (pos[b] - pos[a])) / r

            up = (np.mean([pos[a] for a in range(4) if not s[a]], axis=0) -
                  np.mean([pos[a] for a in range(4) if s[a]], axis=0))
            if nneg in (1, 3):
                odd = [a for a in range(4) if s[a] == (nneg == 1)][0]
                rest = [a for a in range(4) if a != odd]
                faces = [(vert(odd, rest[0]), vert(odd, rest[1]), vert(odd, rest[2]))]
            else:
                ng = [a for a in range(4) if s[a]]
                ps = [a for a in range(4) if not s[a]]
                q = [vert(ng[0], ps[0]), vert(ng[0], ps[1]), vert(ng[1], ps[1]), vert(ng[1], ps[0])]
                faces = [(q[0], q[1], q[2]), (q[0], q[2], q[3])]
            for (p0, p1, p2) in faces:
                n = np.cross(p1 - p0, p2 - p0)
                if np.dot(n, up) < 0:
                    p1, p2, n = p2, p1, -n
                ln = np.linalg.norm(n)
                tris.append((p0, p1, p2))
                nrms.append(n / ln if ln > 0 else n)
    return np.array(tris, np.float64).reshape(-1, 3, 3), np.array(nrms, np.float64).reshape(-1, 3)


def surrogate_dchi(oracle_mod, r, points, normals, dldp):
    """dL/dchi of Eq. 6 on the grid, through the oracle's splat."""
    vals = -np.sum(np.asarray(dldp, np.float64) * np.asarray(normals, np.float64), axis=1)
    return oracle_mod.splat(r, points, vals[:, None])


def topology(tris, decimals=9):
    """(vertices, edges, faces, edges used by exactly two faces) of a triangle
    soup whose shared vertices coincide exactly."""
    key = np.round(tris.reshape(-1, 3), decimals)
    _, inv = np.unique(key, axis=0, return_inverse=True)
    idx = inv.reshape(-1, 3)
    e = np.sort(np.concatenate([idx[:, [0, 1]], idx[:, [1, 2]], idx[:, [2, 0]]]), axis=1)
    ue, cnt = np.unique(e, axis=0, return_counts=True)
    return int(inv.max() + 1), len(ue), len(idx), int(np.sum(cnt == 2))

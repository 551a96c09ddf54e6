"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests and the bench.

This module holds no arithmetic of the method: it only makes meshes (vertex and triangle
arrays), random coefficient vectors and point samples of a heat-kernel datum.  The paper's
experiments (Section 5) use a cube-shaped domain and a crankshaft mesh that is not public;
the meshes here stand in for them.

* ``cube_mesh(n_a, split)``: surface of [0,1]^3, every face an n_a x n_a grid of squares.
  ``split="diag"`` cuts each square by the diagonal from (i,j) to (i+1,j+1) into 2 triangles
  (12 n_a^2 triangles: 192, 768, 3072, 12288, 49152 for n_a = 4, 8, 16, 32, 64);
  ``split="cross"`` adds the square's centre and cuts it into 4 triangles (24 n_a^2:
  1536, 6144 for n_a = 8, 16).  Triangles are oriented counter-clockwise seen from outside,
  so the right-hand normal points out of the cube (the sign convention of Section 2).
* ``cube_sphere_mesh``: the same mesh centred at the origin with its vertices pushed out
  radially to radius 0.5 (stands in for an "icosphere" with those triangle counts).
"""
from __future__ import annotations

import numpy as np

# Face frames (origin, e_u, e_v) of the unit cube with e_u x e_v = outward normal.
_FACES = (
    ((0, 0, 0), (0, 0, 1), (0, 1, 0)),  # x = 0, normal -x
    ((1, 0, 0), (0, 1, 0), (0, 0, 1)),  # x = 1, normal +x
    ((0, 0, 0), (1, 0, 0), (0, 0, 1)),  # y = 0, normal -y
    ((0, 1, 0), (0, 0, 1), (1, 0, 0)),  # y = 1, normal +y
    ((0, 0, 0), (0, 1, 0), (1, 0, 0)),  # z = 0, normal -z
    ((0, 0, 1), (1, 0, 0), (0, 1, 0)),  # z = 1, normal +z
)


def cube_mesh(n_a: int, split: str = "diag"):
    """Return (vertices float64 [N_v,3], triangles int32 [E_x,3]) of the unit cube surface."""
    if n_a < 1:
        raise ValueError("n_a must be >= 1")
    if split not in ("diag", "cross"):
        raise ValueError("split must be 'diag' or 'cross'")
    s = 2  # lattice refinement so that square centres are integer points
    key_to_idx: dict[tuple[int, int, int], int] = {}
    verts: list[tuple[int, int, int]] = []

    def vid(p):
        k = (int(p[0]), int(p[1]), int(p[2]))
        i = key_to_idx.get(k)
        if i is None:
            i = len(verts)
            key_to_idx[k] = i
            verts.append(k)
        return i

    tris: list[tuple[int, int, int]] = []
    for o, eu, ev in _FACES:
        o = np.array(o) * n_a * s
        eu = np.array(eu)
        ev = np.array(ev)
        for i in range(n_a):
            for j in range(n_a):
                p00 = vid(o + s * (i * eu + j * ev))
                p10 = vid(o + s * ((i + 1) * eu + j * ev))
                p11 = vid(o + s * ((i + 1) * eu + (j + 1) * ev))
                p01 = vid(o + s * (i * eu + (j + 1) * ev))
                if split == "diag":
                    tris.append((p00, p10, p11))
                    tris.append((p00, p11, p01))
                else:
                    c = vid(o + s * (i * eu + j * ev) + (eu + ev))
                    tris.append((p00, p10, c))
                    tris.append((p10, p11, c))
                    tris.append((p11, p01, c))
                    tris.append((p01, p00, c))
    V = np.array(verts, dtype=np.float64) / float(n_a * s)
    T = np.array(tris, dtype=np.int32)
    return V, T


def cube_sphere_mesh(n_a: int, split: str = "diag", radius: float = 0.5):
    """Cube mesh centred at the origin with vertices projected radially to ``radius``."""
    V, T = cube_mesh(n_a, split)
    P = V - 0.5
    P = radius * P / np.linalg.norm(P, axis=1, keepdims=True)
    return np.ascontiguousarray(P), T


def random_density(n_steps: int, n_cols: int, nrhs: int = 1, seed: int = 1234):
    """N(0,1) coefficient vectors, layout [nrhs][n_steps][n_cols] (time-major per rhs)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nrhs, n_steps, n_cols))


def heat_source_datum(vertices, T: float, n_steps: int, sources, alpha: float = 1.0):
    """Nodal Dirichlet datum g = sum_s G_alpha(x - y_s, t - t0_s), sampled at every vertex and
    at the midpoint of every time step (piecewise constant in time, piecewise linear in space).

    ``sources`` is a list of (y (3,), t0).  Layout [n_steps][N_v].  This is input generation: it
    samples the closed-form datum of Section 5 (Eq. dirdata), it does not project it.
    """
    V = np.asarray(vertices, dtype=np.float64)
    h = T / n_steps
    tm = (np.arange(n_steps) + 0.5) * h
    g = np.zeros((n_steps, V.shape[0]))
    for y, t0 in sources:
        r2 = np.sum((V - np.asarray(y, dtype=np.float64)) ** 2, axis=1)
        dt = tm - t0
        for k in range(n_steps):
            if dt[k] > 0:
                g[k] += (4 * np.pi * alpha * dt[k]) ** -1.5 * np.exp(-r2 / (4 * alpha * dt[k]))
    return g


def shell_sources(n: int, center=(0.5, 0.5, 0.5), rmin=1.2, rmax=2.0, t0_range=(-0.5, -0.05), seed=2025):
    """``n`` heat sources with |y - c| ~ U[rmin, rmax], direction uniform on S^2, t0 ~ U[t0_range]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        rad = rng.uniform(rmin, rmax)
        t0 = rng.uniform(*t0_range)
        out.append((np.asarray(center) + rad * d, t0))
    return out


def sample_triangles(n_triangles: int, count: int, seed: int = 7):
    """A sorted, seeded sample of distinct triangle indices (targets for sampled parity checks)."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n_triangles, size=min(count, n_triangles), replace=False)).astype(np.int32)

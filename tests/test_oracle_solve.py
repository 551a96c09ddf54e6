"""Pins of the oracle's solve (Section 2, Eq. 02:linear:system; Section 5, Eq. dirdata):
GMRES agrees with the exact block forward substitution, and for the Dirichlet datum
u = G_alpha(x - y*, t) with y* outside the domain the computed Neumann datum converges to the
closed-form trace w = alpha du/dn = -(x - y*).n G_alpha(x - y*, t) / (2 t) under refinement
with h_t ~ h_x^2."""
import math

import numpy as np
import pytest

import oracle as O
from oracle.solve import forward_substitution, gmres
from paper_2106_15911_gb300.inputs import cube_mesh


def _heat(x, y, t, alpha=1.0):
    r2 = np.sum((x - y) ** 2, axis=-1)
    return np.where(t > 0, (4 * math.pi * alpha * np.maximum(t, 1e-300)) ** -1.5 * np.exp(-r2 / (4 * alpha * np.maximum(t, 1e-300))), 0.0)


def _l2_projection(V, T, Tend, Et, ystar):
    """g_h: per step, p1-in-space L2 projection of the step mean of g (Section 2, after the
    Galerkin formulation).  Degree-5 Gauss (collapsed 3x3) per triangle, 4-point Gauss in time."""
    nv, nt = V.shape[0], T.shape[0]
    xq, wq = O.gauss_legendre01(3)
    s1 = np.repeat(xq, 3)
    s2 = np.repeat(xq, 3) * np.tile(xq, 3)
    ww = np.repeat(wq, 3) * np.tile(wq, 3) * np.repeat(xq, 3)
    lam = np.stack([1 - s1, s1 - s2, s2], axis=1)  # barycentric of the points
    xt, wt = O.gauss_legendre01(4)
    h = Tend / Et
    Mp1 = np.zeros((nv, nv))
    rhs = np.zeros((Et, nv))
    for x in range(nt):
        P = V[T[x]]
        J = np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[1]))
        pts = lam @ P
        for a in range(3):
            for b in range(3):
                Mp1[T[x][a], T[x][b]] += np.sum(ww * J * lam[:, a] * lam[:, b])
        for k in range(Et):
            gv = sum(wt[i] * _heat(pts, ystar, (k + xt[i]) * h) for i in range(4))  # step mean of g
            for a in range(3):
                rhs[k, T[x][a]] += np.sum(ww * J * lam[:, a] * gv)
    return np.linalg.solve(Mp1, rhs.T).T


def _solve_dirichlet(n_a, Et, Tend, ystar):
    V, T = cube_mesh(n_a)
    h = Tend / Et
    A = O.assemble_V(V, T, h, nd=Et)
    B = O.assemble_K(V, T, h, nd=Et)
    M = O.assemble_M(V, T, h)
    g = _l2_projection(V, T, Tend, Et, ystar)
    b = 0.5 * (g @ M.T) + O.toeplitz_apply(B, g)
    return V, T, A, b


def test_gmres_matches_forward_substitution():
    ystar = np.array([1.5, 1.5, 1.5])
    V, T, A, b = _solve_dirichlet(2, 16, 1.0, ystar)
    w_exact = forward_substitution(A, b)
    w, it, hist = gmres(lambda x: O.toeplitz_apply(A, x), b, tol=1e-8, restart=50)
    res = np.linalg.norm(b - O.toeplitz_apply(A, w)) / np.linalg.norm(b)
    assert res <= 1e-8
    Et, n = A.shape[0], A.shape[1]
    full = np.zeros((Et * n, Et * n))  # the whole block lower-triangular system
    for k in range(Et):
        for j in range(k + 1):
            full[k * n:(k + 1) * n, j * n:(j + 1) * n] = A[k - j]
    cond = np.linalg.cond(full)
    assert np.linalg.norm(w - w_exact) / np.linalg.norm(w_exact) <= 1e-8 * cond
    assert 5 < it < 200


@pytest.mark.slow
def test_neumann_datum_converges_to_closed_form_trace():
    ystar = np.array([1.5, 1.5, 1.5])
    Tend = 1.0
    errs = []
    for n_a, Et in ((1, 4), (2, 16), (4, 64)):
        V, T, A, b = _solve_dirichlet(n_a, Et, Tend, ystar)
        w = forward_substitution(A, b)
        h = Tend / Et
        cen = V[T].mean(axis=1)
        nrm = np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]])
        area = 0.5 * np.linalg.norm(nrm, axis=1)
        nrm /= (2 * area)[:, None]
        tm = (np.arange(Et) + 0.5) * h
        ex = np.array([-np.sum((cen - ystar) * nrm, axis=1) * _heat(cen, ystar, t) / (2 * t) for t in tm])
        wgt = h * area[None, :]
        errs.append(math.sqrt(np.sum(wgt * (w - ex) ** 2) / np.sum(wgt * ex ** 2)))
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 0.2 and errs[1] / errs[2] > 1.4, errs

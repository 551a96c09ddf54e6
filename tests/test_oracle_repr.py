"""Pins of the oracle's representation formula u = V~ w - W u (Section 2) at interior and exterior
space-time points: its two time antiderivatives against adaptive quadrature, and the formula
itself against the closed-form solution it must reproduce as the boundary element mesh is refined
(u = G(x - y0, t) with the source outside the domain: the exact value inside, zero outside, by
Green's representation theorem for the heat equation)."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O
from paper_2106_15911_gb300.inputs import cube_mesh, heat_source_datum


def _G(r, s, alpha):
    return (4 * math.pi * alpha * s) ** -1.5 * math.exp(-r * r / (4 * alpha * s))


@pytest.mark.parametrize("r,s,alpha", [(0.05, 0.01, 1.0), (0.3, 0.5, 1.0), (1.2, 0.2, 0.5), (0.8, 3.0, 2.0)])
def test_time_antiderivatives(r, s, alpha):
    g1 = integrate.quad(lambda q: _G(r, q, alpha), 0, s, epsabs=0, epsrel=1e-13, limit=200)[0]
    h1 = integrate.quad(lambda q: _G(r, q, alpha) / (2 * q), 0, s, epsabs=0, epsrel=1e-13, limit=200)[0]
    assert O.G1(r, s, alpha) == pytest.approx(g1, rel=1e-11)
    assert O.H1(r, s, alpha) == pytest.approx(h1, rel=1e-11)
    assert O.H1(r, 0.0, alpha) == 0.0 and O.G1(r, -1.0, alpha) == 0.0


def _traces(V, T, Et, y0, alpha=1.0):
    """Element data of u = G(x - y0, t): the Neumann trace w = alpha du/dn = -(x - y0).n / (2 t) u
    at triangle centroids and step midpoints, the Dirichlet datum at the vertices and midpoints."""
    h = 1.0 / Et
    tm = (np.arange(Et) + 0.5) * h
    P = V[T]
    c = P.mean(axis=1)
    n = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    n /= np.linalg.norm(n, axis=1)[:, None]
    d = c - np.asarray(y0)
    r2 = np.sum(d * d, axis=1)
    dn = np.sum(d * n, axis=1)
    w = np.array([-dn / (2 * t) * (4 * np.pi * alpha * t) ** -1.5 * np.exp(-r2 / (4 * alpha * t)) for t in tm])
    g = heat_source_datum(V, 1.0, Et, [(y0, 0.0)], alpha)
    return w, g


def test_representation_formula_converges_to_the_solution_inside_and_zero_outside():
    y0 = (1.5, 1.5, 1.5)
    x_in, x_out, t = (0.5, 0.45, 0.55), (-0.6, 0.5, 0.4), 1.0
    exact_in = _G(math.dist(x_in, y0), t, 1.0)
    pts = np.array([[*x_in, t], [*x_out, t]])
    err_in, err_out = [], []
    for n_a, Et in ((2, 4), (4, 16), (8, 64)):
        V, T = cube_mesh(n_a)
        w, g = _traces(V, T, Et, y0)
        P = O.make_problem(V, T, 1.0, Et, n_r=6)
        u = O.repr_eval(P, w, g, pts)
        err_in.append(abs(u[0] - exact_in))
        err_out.append(abs(u[1]))
    assert err_in[2] < err_in[1] < err_in[0] and err_in[2] < 0.03 * exact_in, (err_in, exact_in)
    assert err_out[2] < err_out[1] < err_out[0] and err_out[2] < 0.03 * exact_in, err_out


def test_representation_formula_is_causal_and_linear():
    V, T = cube_mesh(2)
    Et = 8
    rng = np.random.default_rng(5)
    w = rng.standard_normal((Et, T.shape[0]))
    g = rng.standard_normal((Et, V.shape[0]))
    P = O.make_problem(V, T, 1.0, Et)
    pts = np.array([[0.5, 0.5, 0.5, 0.0], [0.5, 0.5, 0.5, 0.3], [0.4, 0.6, 0.5, 0.7]])
    u = O.repr_eval(P, w, g, pts)
    assert u[0] == 0.0
    # data after the point's time do not contribute
    w2, g2 = w.copy(), g.copy()
    w2[3:] = 7.0
    g2[3:] = -3.0
    assert O.repr_eval(P, w2, g2, pts[1:2])[0] == u[1]
    # linear in (w, g); V~ w alone with g = None
    uw = O.repr_eval(P, w, None, pts)
    ug = O.repr_eval(P, np.zeros_like(w), g, pts)
    assert np.allclose(uw + ug, u, rtol=1e-13, atol=1e-16)

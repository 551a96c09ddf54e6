"""Pins of the oracle's S2M / L2T moments (Section 3.4, Eq. s2m and l2t) against exact
integration that shares nothing with the oracle's quadrature.

* Spatial moments: the integrand T_kappa((y - c) / h) (single layer) or
  alpha n . grad_y T_kappa((y - c) / h) phi_v(y) (double layer) is a polynomial in the barycentric
  coordinates of the triangle; each monomial integrates in closed form,
  int lambda_1^i lambda_2^j lambda_3^k dA = 2 |x| i! j! k! / (i + j + k + 2)!.
* Time moments: integrals of the Lagrange basis over a step reproduce the integral of every
  polynomial of degree <= m_t through the interpolation nodes, and sum to the step length.

A wrong Jacobian, box scaling, vertex-to-coordinate map, normal orientation or integration range
fails one of these."""
from math import factorial

import numpy as np
import pytest

import oracle as O
from paper_2106_15911_gb300.inputs import cube_sphere_mesh

# ---- polynomials in the barycentric coordinates (lambda_1, lambda_2, lambda_3) ----------------


def _padd(p, q, s=1.0):
    r = dict(p)
    for k, v in q.items():
        r[k] = r.get(k, 0.0) + s * v
    return r


def _pmul(p, q):
    r = {}
    for (a1, b1, c1), v in p.items():
        for (a2, b2, c2), w in q.items():
            k = (a1 + a2, b1 + b2, c1 + c2)
            r[k] = r.get(k, 0.0) + v * w
    return r


def _pscale(p, s):
    return {k: s * v for k, v in p.items()}


ONE = {(0, 0, 0): 1.0}


def _affine(vals):
    """The linear function with values vals[v] at the three vertices: sum_v vals[v] lambda_v."""
    return {(1, 0, 0): vals[0], (0, 1, 0): vals[1], (0, 0, 1): vals[2]}


def _cheb(u, n, second_kind=False):
    """[T_0(u) .. T_n(u)] (or U_0 .. U_n) as polynomials, by the three-term recurrence."""
    out = [ONE, _pscale(u, 2.0 if second_kind else 1.0)]
    while len(out) <= n:
        out.append(_padd(_pscale(_pmul(u, out[-1]), 2.0), out[-2], -1.0))
    return out[: n + 1]


def _integrate(p, area):
    return sum(v * 2.0 * area * factorial(i) * factorial(j) * factorial(k) / factorial(i + j + k + 2)
               for (i, j, k), v in p.items())


def _exact_space_moments(P, V, T, x, cen, hp, op, alpha):
    A, B, C = (V[T[x, v]] for v in range(3))
    cr = np.cross(B - A, C - A)
    area = 0.5 * np.linalg.norm(cr)
    n = cr / np.linalg.norm(cr)
    m = P.m_x
    u = [_affine([(A[c] - cen[c]) / hp, (B[c] - cen[c]) / hp, (C[c] - cen[c]) / hp]) for c in range(3)]
    Tc = [_cheb(u[c], m) for c in range(3)]
    Uc = [_cheb(u[c], m, second_kind=True) for c in range(3)]

    def dT(c, k):  # T_k'(u) = k U_{k-1}(u)
        return _pscale(Uc[c][k - 1], float(k)) if k > 0 else {}

    lam = [{(1, 0, 0): 1.0}, {(0, 1, 0): 1.0}, {(0, 0, 1): 1.0}]
    out = []
    for (k0, k1, k2) in O.multi_indices(m):
        if op == 0:
            out.append(_integrate(_pmul(_pmul(Tc[0][k0], Tc[1][k1]), Tc[2][k2]), area))
            continue
        g = [_pmul(_pmul(dT(0, k0), Tc[1][k1]), Tc[2][k2]),
             _pmul(_pmul(Tc[0][k0], dT(1, k1)), Tc[2][k2]),
             _pmul(_pmul(Tc[0][k0], Tc[1][k1]), dT(2, k2))]
        dn = {}
        for c in range(3):
            dn = _padd(dn, g[c], alpha * n[c] / hp)
        out.append([_integrate(_pmul(dn, lam[v]), area) for v in range(3)])
    return np.array(out)


def _single_triangle(seed):
    rng = np.random.default_rng(seed)
    V = rng.uniform(-0.5, 0.5, (3, 3))
    return V, np.array([[0, 1, 2]], dtype=np.int32)


@pytest.mark.parametrize("m_x", [0, 3, 6, 9])
@pytest.mark.parametrize("op", [0, 1])
def test_space_moments_are_exact_polynomial_integrals(m_x, op):
    alpha = 0.7
    cases = []
    V1, T1 = _single_triangle(5)
    cases.append((V1, T1, 0, np.array([0.05, -0.1, 0.2]), 0.6))
    V2, T2 = cube_sphere_mesh(2)
    cases.append((V2, T2, 7, V2[T2[7]].mean(axis=0) + np.array([0.1, -0.05, 0.02]), 0.4))
    cases.append((V2, T2, 30, V2[T2[30]].mean(axis=0) - np.array([0.2, 0.1, -0.15]), 0.9))
    for V, T, x, cen, hp in cases:
        P = O.make_problem(V, T, 1.0, 4, alpha=alpha, m_x=m_x)
        got = O.space_moments(P, x, cen, hp, op)
        ref = _exact_space_moments(P, np.asarray(V, float), np.asarray(T), x, cen, hp, op, alpha)
        scale = np.max(np.abs(ref))
        if scale == 0:  # double layer at m_x = 0: grad T_0 = 0
            assert op == 1 and m_x == 0 and not np.any(got)
            continue
        assert np.max(np.abs(got - ref)) <= 1e-12 * scale, (m_x, op, x, np.max(np.abs(got - ref)) / scale)


def test_space_moments_detect_a_reversed_triangle():
    """The double-layer moments follow the triangle's orientation (the normal of its vertex order);
    the single-layer moments do not depend on it."""
    V, T = _single_triangle(11)
    Tr = T[:, ::-1].copy()
    cen, hp = np.array([0.0, 0.1, -0.1]), 0.7
    P, Pr = O.make_problem(V, T, 1.0, 4, m_x=4), O.make_problem(V, Tr, 1.0, 4, m_x=4)
    assert np.allclose(O.space_moments(P, 0, cen, hp, 0), O.space_moments(Pr, 0, cen, hp, 0), rtol=0, atol=1e-14)
    d, dr = O.space_moments(P, 0, cen, hp, 1), O.space_moments(Pr, 0, cen, hp, 1)
    assert np.allclose(d, -dr[:, ::-1], rtol=0, atol=1e-13)


@pytest.mark.parametrize("m_t", [0, 1, 4, 7])
def test_time_moments_reproduce_polynomial_integrals(m_t):
    """sum_a L_{J,a}(t) t_a^p = t^p for p <= m_t (t_a the interpolation nodes of J), so the moments
    of a step (lo, lo + h] inside J reproduce int t^p over it; p = 0 is the step length."""
    jlo, jhi = 0.25, 1.75
    mid, half = 0.5 * (jlo + jhi), 0.5 * (jhi - jlo)
    nodes = np.array([mid + half * O.cheb_node(a, m_t) for a in range(m_t + 1)])
    for lo, h in [(0.25, 0.1875), (1.0, 0.75), (0.3, 0.01)]:
        mom = np.array([O.time_moment(a, m_t, jlo, jhi, lo, h) for a in range(m_t + 1)])
        for p in range(m_t + 1):
            exact = ((lo + h) ** (p + 1) - lo ** (p + 1)) / (p + 1)
            assert abs(mom @ nodes ** p - exact) <= 1e-13 * max(1.0, abs(exact)), (m_t, lo, h, p)
    # degree m_t + 1 is not reproduced: the error is the integral of the node polynomial
    # prod_a (t - t_a), which the check must see
    lo, h = 1.0, 0.75
    mom = np.array([O.time_moment(a, m_t, jlo, jhi, lo, h) for a in range(m_t + 1)])
    p = m_t + 1
    err = ((lo + h) ** (p + 1) - lo ** (p + 1)) / (p + 1) - mom @ nodes ** p
    node_poly = np.polynomial.polynomial.polyfromroots(nodes)
    integ = np.polynomial.polynomial.polyint(node_poly)
    expect = np.polynomial.polynomial.polyval(lo + h, integ) - np.polynomial.polynomial.polyval(lo, integ)
    assert abs(expect) > 1e-6
    assert abs(err - expect) <= 1e-12 * max(1.0, abs(expect))

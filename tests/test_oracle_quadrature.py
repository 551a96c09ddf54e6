"""Pins of the oracle's spatial quadrature (the nearfield rule chosen where the paper defers to
another publication, Section 3.4 after Eq. eval_sl_nf_block).

* Gauss-Legendre and the collapsed triangle rule integrate polynomials exactly (closed-form
  monomial integrals over a triangle).
* The Sauter-Schwab transformations for identical, edge- and vertex-adjacent triangles
  integrate smooth kernels like the plain product rule (so the regions and Jacobians are right).
* For the weakly singular Laplace single layer 1/(4 pi r) and the Laplace double layer
  (x-y).n_y/(4 pi r^3) (the leading terms of V_h at d = 0 and K_h at d = 0) they match the
  closed-form potentials of a flat triangle (Wilton et al. 1984; Van Oosterom & Strackee 1983),
  integrated over the target triangle by refined quadrature.
"""
import math

import numpy as np
import pytest

import oracle as O


# ---------------------------------------------------------------------------------------------
def test_gauss_legendre_exact():
    for n in (1, 2, 3, 5, 8, 13, 20):
        x, w = O.gauss_legendre01(n)
        assert np.all((x > 0) & (x < 1))
        for k in range(2 * n):
            assert np.dot(w, x ** k) == pytest.approx(1.0 / (k + 1), rel=1e-13)


def _mono_tri(P, a, b, c):
    """int over triangle P of lambda0^a lambda1^b lambda2^c = 2A a! b! c! / (a+b+c+2)!"""
    A = 0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))
    return 2 * A * math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 2)


def _int_coord_poly(P, powers):
    """int over triangle P of prod_c x_c^{powers[c]} by expanding x = sum_i lambda_i P_i."""
    # expand each coordinate power through the multinomial theorem in barycentric monomials
    from itertools import product

    terms = {(0, 0, 0): 1.0}
    for c, pw in enumerate(powers):
        for _ in range(pw):
            new = {}
            for (a, b, cc), v in terms.items():
                for i, coef in enumerate(P[:, c]):
                    key = (a + (i == 0), b + (i == 1), cc + (i == 2))
                    new[key] = new.get(key, 0.0) + v * coef
            terms = new
    return sum(v * _mono_tri(P, *k) for k, v in terms.items())


# six points; every listed pair of triangles meets only in its shared vertices (no intersections)
V6 = np.array([[0, 0, 0], [1, 0, 0], [0.3, 0.9, 0], [0.4, -0.2, 0.8], [-0.7, 0.1, -0.5], [-0.4, -0.6, 0.3]], float)
PAIRS = [((0, 1, 2), (0, 1, 2)), ((0, 1, 2), (1, 0, 3)), ((0, 1, 2), (0, 4, 5)), ((0, 1, 2), (2, 5, 3)),
         ((0, 1, 2), (3, 4, 5))]


@pytest.mark.parametrize("tx,ty", PAIRS)
def test_regular_rule_exact_for_polynomials(tx, ty):
    poly = (0.7, 1.3, -0.9, 0.0)  # c0 + c1 x0 y1 + c2 x2^2 y0 y1
    X, Y = V6[list(tx)], V6[list(ty)]
    exact = (poly[0] * _int_coord_poly(X, (0, 0, 0)) * _int_coord_poly(Y, (0, 0, 0))
             + poly[1] * _int_coord_poly(X, (1, 0, 0)) * _int_coord_poly(Y, (0, 1, 0))
             + poly[2] * _int_coord_poly(X, (0, 0, 2)) * _int_coord_poly(Y, (1, 1, 0)))
    got = O.pair_integral(V6, tx, ty, O.KIND_POLY, 3, use_ss=False, poly=poly)
    assert got == pytest.approx(exact, rel=1e-13)


@pytest.mark.parametrize("tx,ty", PAIRS[:4])
def test_sauter_schwab_matches_product_rule_on_smooth_kernels(tx, ty):
    poly = (0.7, 1.3, -0.9, 0.5)  # includes a Gaussian of |x - y|
    ref = O.pair_integral(V6, tx, ty, O.KIND_POLY, 14, use_ss=False, poly=poly)
    ss = O.pair_integral(V6, tx, ty, O.KIND_POLY, 9, use_ss=True, poly=poly)
    assert ss == pytest.approx(ref, rel=1e-12)
    # polynomial kernels: the transformed integrands are polynomials, so the rule is exact
    poly0 = (0.7, 1.3, -0.9, 0.0)
    ref0 = O.pair_integral(V6, tx, ty, O.KIND_POLY, 6, use_ss=False, poly=poly0)
    assert O.pair_integral(V6, tx, ty, O.KIND_POLY, 6, use_ss=True, poly=poly0) == pytest.approx(ref0, rel=1e-13)


# ---- closed-form potentials of a flat triangle -------------------------------------------------
def lap_sl_potential(x, P):
    """int_T 1/|x - y| dy for a flat triangle P (3x3), Wilton et al. (1984), eq. for a constant
    source: sum over edges of P0 ln((R+ + l+)/(R- + l-)) - |d| sum [atan(..+) - atan(..-)]."""
    n = np.cross(P[1] - P[0], P[2] - P[0])
    n /= np.linalg.norm(n)
    d = np.dot(x - P[0], n)
    rho = x - d * n
    tot = 0.0
    for i in range(3):
        a, b = P[i], P[(i + 1) % 3]
        lhat = (b - a) / np.linalg.norm(b - a)
        uhat = np.cross(lhat, n)
        lp, lm = np.dot(b - rho, lhat), np.dot(a - rho, lhat)
        P0 = np.dot(a - rho, uhat)
        Rp, Rm = np.linalg.norm(x - b), np.linalg.norm(x - a)
        R0sq = P0 * P0 + d * d
        if abs(P0) > 1e-14:
            tot += P0 * math.log((Rp + lp) / (Rm + lm))
        if abs(d) > 0:
            tot -= abs(d) * (math.atan(P0 * lp / (R0sq + abs(d) * Rp)) - math.atan(P0 * lm / (R0sq + abs(d) * Rm)))
    return tot


def solid_angle(x, P):
    """int_T (x - y).n_y / |x - y|^3 dy: the solid angle of T seen from x, positive on the side the
    normal points to (Van Oosterom & Strackee 1983, with R_i = x - P_i)."""
    R = [x - P[i] for i in range(3)]
    Rn = [np.linalg.norm(r) for r in R]
    num = np.dot(R[0], np.cross(R[1], R[2]))
    den = Rn[0] * Rn[1] * Rn[2] + np.dot(R[0], R[1]) * Rn[2] + np.dot(R[0], R[2]) * Rn[1] + np.dot(R[1], R[2]) * Rn[0]
    return 2.0 * math.atan2(num, den)


def _tri_points(P, level, n):
    """points and weights of a collapsed Gauss rule on 4^level congruent subtriangles of P."""
    x, w = O.gauss_legendre01(n)
    s1 = np.repeat(x, n)
    s2 = np.repeat(x, n) * np.tile(x, n)
    ww = np.repeat(w, n) * np.tile(w, n) * np.repeat(x, n)
    tris = [np.asarray(P, float)]
    for _ in range(level):
        nxt = []
        for T in tris:
            m01, m12, m20 = (T[0] + T[1]) / 2, (T[1] + T[2]) / 2, (T[2] + T[0]) / 2
            nxt += [np.array([T[0], m01, m20]), np.array([m01, T[1], m12]), np.array([m20, m12, T[2]]),
                    np.array([m12, m20, m01])]
        tris = nxt
    pts, wts = [], []
    for T in tris:
        J = np.linalg.norm(np.cross(T[1] - T[0], T[2] - T[1]))
        pts.append(T[0] + np.outer(s1, T[1] - T[0]) + np.outer(s2, T[2] - T[1]))
        wts.append(ww * J)
    return np.vstack(pts), np.concatenate(wts)


def test_closed_form_potentials_against_brute_force():
    P = V6[[0, 1, 2]]
    for x in (np.array([0.2, 0.3, 0.4]), np.array([1.3, -0.4, -0.2]), np.array([0.35, 0.25, 0.05])):
        pts, w = _tri_points(P, 3, 12)
        r = np.linalg.norm(x - pts, axis=1)
        n = np.cross(P[1] - P[0], P[2] - P[0])
        n /= np.linalg.norm(n)
        assert lap_sl_potential(x, P) == pytest.approx(np.sum(w / r), rel=1e-9)
        assert solid_angle(x, P) == pytest.approx(np.sum(w * ((x - pts) @ n) / r ** 3), rel=1e-7)


SING_PAIRS = [
    ((0, 1, 2), (0, 1, 2)),  # identical
    ((0, 1, 2), (1, 0, 6)),  # common edge, coplanar
    ((0, 1, 2), (1, 0, 3)),  # common edge, bent
    ((0, 1, 2), (0, 4, 5)),  # common vertex
    ((0, 1, 2), (2, 7, 5)),  # common vertex
]
V8 = np.vstack([V6, [[0.5, -0.7, 0.0]], [[0.2, 1.6, 0.4]]])


def _outer(fun, X, Y):
    """int over X of fun(x, Y) on 4^3, 4^4 and 4^5 subtriangles, Aitken-extrapolated: the
    potentials have log-type derivatives at edges and vertices, so the refined rule converges
    only algebraically (O(h^2) or O(h^3) depending on the pair)."""
    vals = []
    for lev in (3, 4, 5):
        pts, w = _tri_points(X, lev, 6)
        vals.append(sum(wi * fun(p, Y) for p, wi in zip(pts, w)))
    d1, d2 = vals[1] - vals[0], vals[2] - vals[1]
    if abs(d2) < 1e-16 * abs(vals[2]) or d1 == d2:
        return vals[2]
    return vals[2] - d2 * d2 / (d2 - d1)


@pytest.mark.parametrize("tx,ty", SING_PAIRS)
def test_sauter_schwab_laplace_single_layer(tx, ty):
    X, Y = V8[list(tx)], V8[list(ty)]
    ref = _outer(lap_sl_potential, X, Y) / (4 * math.pi)
    got = O.pair_integral(V8, tx, ty, O.KIND_LAPSL, 24, use_ss=True)
    assert got == pytest.approx(ref, rel=2e-9)


@pytest.mark.parametrize("tx,ty", SING_PAIRS[1:])
def test_sauter_schwab_laplace_double_layer(tx, ty):
    X, Y = V8[list(tx)], V8[list(ty)]
    ref = _outer(solid_angle, X, Y) / (4 * math.pi)
    got = O.pair_integral(V8, tx, ty, O.KIND_LAPDL, 24, use_ss=True)
    assert got == pytest.approx(ref, rel=1e-7, abs=1e-12)


def _cube_singular_pairs():
    from paper_2106_15911_gb300.inputs import cube_mesh

    V, T = cube_mesh(2)
    out = {}
    for x in range(T.shape[0]):
        for y in range(T.shape[0]):
            sh = len(set(T[x]) & set(T[y]))
            n_same = abs(np.dot(np.cross(V[T[x][1]] - V[T[x][0]], V[T[x][2]] - V[T[x][0]]),
                                np.cross(V[T[y][1]] - V[T[y][0]], V[T[y][2]] - V[T[y][0]])))
            key = (sh, n_same > 1e-12)
            if sh > 0 and key not in out:
                out[key] = (T[x], T[y])
    return V, list(out.values())


def test_sauter_schwab_converges_for_heat_kernels():
    """Self-convergence of the singular rule on the time-integrated heat kernels at d = 0, 1 for
    the pair classes of the cube meshes (identical, coplanar and right-angled neighbours)."""
    V, pairs = _cube_singular_pairs()
    assert len(pairs) >= 4
    for tx, ty in pairs:
        for kind in (O.KIND_V, O.KIND_K):
            for d in (0, 1):
                hi = np.atleast_1d(O.pair_integral(V, tx, ty, kind, 14, use_ss=True, d=d, h=1.0 / 64))
                lo = np.atleast_1d(O.pair_integral(V, tx, ty, kind, 8, use_ss=True, d=d, h=1.0 / 64))
                scale = np.max(np.abs(hi)) + 1e-300
                assert np.max(np.abs(hi - lo)) / scale < 1e-6, (tx, ty, kind, d)

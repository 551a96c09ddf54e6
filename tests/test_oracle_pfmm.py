"""Pins of the oracle's pFMM (Section 3): the expansion ingredients reproduce what they
interpolate (Eq. kernel_approx, exp_coeffs_1d, temp_m2m, st_m2m), the nearfield part equals
the dense matrix restricted to the nearfield blocks (Eq. eval_sl_nf_block), the sampled-target
mode returns the same rows as a full apply, and the approximation error against the dense
Galerkin product decreases with the expansion degrees (Section 3.1, after Eq. exp_coeffs_1d)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2106_15911_gb300.inputs import cube_mesh, random_density


def _T(k, x):
    return math.cos(k * math.acos(max(-1.0, min(1.0, x))))


def test_lagrange_cardinal_and_partition_of_unity():
    m, lo, hi = 5, 0.3, 0.8
    nodes = [0.5 * (lo + hi) + 0.5 * (hi - lo) * O.cheb_node(k, m) for k in range(m + 1)]
    for b in range(m + 1):
        for k in range(m + 1):
            assert O.lagrange(b, m, lo, hi, nodes[k]) == pytest.approx(1.0 if b == k else 0.0, abs=1e-13)
    for t in np.linspace(lo, hi, 7):
        assert sum(O.lagrange(b, m, lo, hi, t) for b in range(m + 1)) == pytest.approx(1.0, abs=1e-13)


@pytest.mark.parametrize("r,dab", [(0.0, 1.0), (2.0, 1.0), (-4.0, 3.0), (6.0, 8.0)])
def test_E1_expansion_reproduces_the_gaussian(r, dab):
    """sum_{k,l} E_{k,l}(r, d) T_l(x) T_k(y) -> exp(-(r + x - y)^2 / d) on [-1,1]^2."""
    rng = np.random.default_rng(3)
    pts = rng.uniform(-1, 1, size=(6, 2))
    errs = []
    for m in (4, 8, 18):
        E = np.array([[O.E1(k, l, r, dab, m) for l in range(m + 1)] for k in range(m + 1)])
        err = 0.0
        for x, y in pts:
            approx = sum(E[k, l] * _T(l, x) * _T(k, y) for k in range(m + 1) for l in range(m + 1))
            err = max(err, abs(approx - math.exp(-(r + x - y) ** 2 / dab)))
        errs.append(err)
    assert errs[0] > errs[1] > errs[2] or errs[2] < 1e-14
    assert errs[2] < 1e-11


def test_temporal_m2m_coefficients_reinterpolate():
    """L_{Ip,ap}(t) = sum_ac q_{ac,ap} L_{Ic,ac}(t) on each half I_c of I_p (exact for degree m)."""
    m = 4
    for c in (0, 1):
        clo, chi = (-1.0, 0.0) if c == 0 else (0.0, 1.0)
        for t in np.linspace(clo, chi, 5):
            for ap in range(m + 1):
                lhs = O.lagrange(ap, m, -1.0, 1.0, t)
                rhs = sum(O.qt(c, ac, ap, m) * O.lagrange(ac, m, clo, chi, t) for ac in range(m + 1))
                assert rhs == pytest.approx(lhs, abs=1e-13)


def test_spatial_m2m_coefficients_reexpand():
    """T_nu((z - cp)/hp) = sum_{kap <= nu} q_{kap,nu} T_kap((z - cc)/hc) for z in the child."""
    m = 6
    cp, hp = 0.5, 0.55  # padded parent
    for cc in (0.25, 0.75):
        hc = 0.3  # padded child
        for z in np.linspace(cc - hc, cc + hc, 6):
            for nu in range(m + 1):
                lhs = _T(nu, (z - cp) / hp)
                rhs = sum(O.qx(k, nu, cc, hc, cp, hp, m) * _T(k, (z - cc) / hc) for k in range(nu + 1))
                assert rhs == pytest.approx(lhs, abs=1e-12)
                for k in range(nu + 1, m + 1):
                    assert abs(O.qx(k, nu, cc, hc, cp, hp, m)) < 1e-13


@pytest.fixture(scope="module")
def cfg1():
    V, T = cube_mesh(4)
    Et, h = 16, 1.0 / 16
    A = O.assemble_V(V, T, h, nd=Et)
    B = O.assemble_K(V, T, h, nd=Et)
    w = random_density(Et, T.shape[0], 1, seed=1234)[0]
    g = random_density(Et, V.shape[0], 1, seed=99)[0]
    return V, T, Et, A, B, w, g


def test_nearfield_part_is_the_dense_nearfield(cfg1):
    V, T, Et, A, B, w, g = cfg1
    P = O.make_problem(V, T, 1.0, Et, m_t=4, m_x=4, c_st=1.0)
    ref = np.zeros((Et, T.shape[0]))
    refk = np.zeros((Et, T.shape[0]))
    for kt in range(Et):
        for jt in range(Et):
            if jt <= kt and (jt // 2) in O.nearfield_list(kt // 2):
                ref[kt] += A[kt - jt] @ w[jt]
                refk[kt] += B[kt - jt] @ g[jt]
    assert np.allclose(O.pfmm_apply(P, 0, w, parts=1), ref, rtol=0, atol=1e-14 * np.abs(ref).max())
    assert np.allclose(O.pfmm_apply(P, 1, g, parts=1), refk, rtol=0, atol=1e-14 * np.abs(refk).max())


def test_sampled_targets_equal_full_rows(cfg1):
    V, T, Et, A, B, w, g = cfg1
    P = O.make_problem(V, T, 1.0, Et, m_t=4, m_x=4, c_st=0.25)
    full = O.pfmm_apply(P, 0, w)
    tg = [3, 50, 51, 190]
    part = O.pfmm_apply(P, 0, w, targets=tg)
    assert np.array_equal(part[:, tg], full[:, tg])
    others = np.setdiff1d(np.arange(T.shape[0]), tg)
    assert np.all(part[:, others] == 0)


@pytest.mark.parametrize("c_st", [1.0, 0.25])
def test_pfmm_error_decreases_with_degree(cfg1, c_st):
    V, T, Et, A, B, w, g = cfg1
    fd = O.toeplitz_apply(A, w)
    errs = []
    for m in (2, 4, 6, 8):
        P = O.make_problem(V, T, 1.0, Et, m_t=m, m_x=m, c_st=c_st)
        f = O.pfmm_apply(P, 0, w)
        errs.append(np.max(np.abs(f - fd)) / np.max(np.abs(fd)))
    assert all(a > b for a, b in zip(errs[:-1], errs[1:])), errs
    assert errs[-1] < (2e-4 if c_st == 1.0 else 2e-6), errs


def test_pfmm_double_layer_error_decreases_with_degree(cfg1):
    V, T, Et, A, B, w, g = cfg1
    fd = O.toeplitz_apply(B, g)
    errs = []
    for m in (2, 4, 6, 8):
        P = O.make_problem(V, T, 1.0, Et, m_t=m, m_x=m, c_st=0.25)
        errs.append(np.max(np.abs(O.pfmm_apply(P, 1, g) - fd)) / np.max(np.abs(fd)))
    assert all(a > b for a, b in zip(errs[:-1], errs[1:])), errs
    assert errs[-1] < 1e-5, errs

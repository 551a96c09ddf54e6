"""Pins of the oracle's heat-kernel time integrals (Section 2, Eq. heat_kernel).

The oracle evaluates the Galerkin time integrals in closed form (second antiderivatives of the
heat kernel in the time difference).  These tests compare them with adaptive quadrature of the
kernel itself, written through a different identity: for uniform steps of length h and offset
d = k - j, the double integral over target and source steps equals the one-dimensional integral
of G(r, s) against the triangle weight max(0, h - |s - d h|).
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O


def _G(r, s, alpha):
    return (4 * math.pi * alpha * s) ** -1.5 * math.exp(-r * r / (4 * alpha * s)) if s > 0 else 0.0


def _tri_weight_integral(fun, d, h, r=None, alpha=1.0):
    lo, hi = max(0.0, (d - 1) * h), (d + 1) * h
    mid = d * h
    cand = [mid]
    if r is not None:  # break points around the kernel's peak in s (at r^2 / (6 alpha)) for small r
        pk = r * r / (6 * alpha)
        cand += [pk * f for f in (0.01, 0.1, 0.3, 1.0, 3.0, 10.0, 100.0, 1e3, 1e4)]
    pts = [p for p in cand if lo < p < hi]
    total = 0.0
    edges = sorted(set([lo] + pts + [hi]))
    for a, b in zip(edges[:-1], edges[1:]):
        total += integrate.quad(lambda s: max(0.0, h - abs(s - mid)) * fun(s), a, b, epsabs=0, epsrel=2e-14,
                                limit=400)[0]
    return total


def _peaked(fun, a, b, peak):
    edges = [a, b]
    if a < peak < b:
        edges = [a, peak, b]
    return sum(integrate.quad(fun, x, y, epsabs=0, epsrel=2e-14, limit=400)[0] for x, y in zip(edges[:-1], edges[1:]))


@pytest.mark.parametrize("alpha", [1.0, 0.37])
@pytest.mark.parametrize("r", [0.003, 0.05, 0.3, 0.9])
@pytest.mark.parametrize("s", [0.002, 0.05, 0.7])
def test_G1_G2_are_antiderivatives(alpha, r, s):
    """G1(r,s) = int_0^s G dq and G2(r,s) = int_0^s (s-q) G dq (repeated integration)."""
    peak = r * r / (6 * alpha)
    g1 = _peaked(lambda q: _G(r, q, alpha), 0.0, s, peak)
    g2 = _peaked(lambda q: (s - q) * _G(r, q, alpha), 0.0, s, peak)
    if g1 > 1e-200:
        assert O.G1(r, s, alpha) == pytest.approx(g1, rel=1e-11)
    if g2 > 1e-200:
        assert O.G2(r, s, alpha) == pytest.approx(g2, rel=1e-10)


@pytest.mark.parametrize("h", [1.0 / 256, 1.0 / 16, 0.5])
@pytest.mark.parametrize("r", [1e-4, 0.01, 0.08, 0.3, 1.0])
@pytest.mark.parametrize("d", [0, 1, 2, 3, 5, 12])
def test_time_V_matches_kernel_integral(h, r, d):
    ref = _tri_weight_integral(lambda s: _G(r, s, 1.0), d, h, r)
    got = O.time_V(r, d, h)
    if ref < 1e-250:
        assert abs(got) < 1e-200
    else:
        assert got == pytest.approx(ref, rel=2e-10, abs=1e-13 * abs(ref) + 1e-300)


@pytest.mark.parametrize("h", [1.0 / 256, 1.0 / 16])
@pytest.mark.parametrize("r", [1e-3, 0.02, 0.1, 0.5])
@pytest.mark.parametrize("d", [0, 1, 2, 3, 7])
def test_time_K_matches_kernel_integral(h, r, d):
    """alpha dG/dn_y = (x-y).n_y G/(2s): the oracle's factor integrates G/(2s) over both steps."""
    ref = _tri_weight_integral(lambda s: _G(r, s, 1.0) / (2 * s) if s > 0 else 0.0, d, h, r)
    got = O.time_K(r, d, h)
    if ref < 1e-250:
        assert abs(got) < 1e-200
    else:
        assert got == pytest.approx(ref, rel=2e-9)


def test_causality_and_small_r_limits():
    h = 0.01
    assert O.time_V(0.1, -1, h) == 0.0 and O.time_K(0.1, -1, h) == 0.0
    # G2 - s/(4 pi alpha r) -> -sqrt(s)/(2 pi^{3/2} alpha^{3/2}) as r -> 0
    for alpha in (1.0, 2.5):
        for s in (1e-3, 0.3):
            lim = -math.sqrt(s) / (2 * math.pi ** 1.5 * alpha ** 1.5)
            assert O.G2t(0.0, s, alpha) == pytest.approx(lim, rel=1e-14)
            assert O.G2t(1e-9, s, alpha) == pytest.approx(lim, rel=1e-7)
    # for d >= 1 the single-layer entry is bounded as r -> 0 and equals the second difference of the limit
    for d in (1, 2, 3):
        lim = -(math.sqrt((d + 1) * h) - 2 * math.sqrt(d * h) + math.sqrt(max(d - 1, 0) * h)) / (2 * math.pi ** 1.5)
        assert O.time_V(0.0, d, h) == pytest.approx(lim, rel=1e-12)


@pytest.mark.parametrize("r", [0.004, 0.02, 0.05])
def test_both_evaluation_branches_agree(r):
    """Near the switch u = 1 both forms (with and without the linear part) give the entry."""
    h = 1.0 / 256
    for d in (1, 2, 3, 6):
        s = [(d + 1) * h, d * h, d * h, (d - 1) * h]
        a = O.G2(r, s[0]) - O.G2(r, s[1]) - O.G2(r, s[2]) + O.G2(r, s[3])
        b = O.G2t(r, s[0]) - O.G2t(r, s[1]) - O.G2t(r, s[2]) + O.G2t(r, s[3])
        assert a == pytest.approx(b, rel=1e-9)
        ka = O.DL2(r, s[0]) - O.DL2(r, s[1]) - O.DL2(r, s[2]) + O.DL2(r, s[3])
        kb = O.DL2t(r, s[0]) - O.DL2t(r, s[1]) - O.DL2t(r, s[2]) + O.DL2t(r, s[3])
        assert ka == pytest.approx(kb, rel=1e-8)


def test_DL2_is_minus_alpha_over_r_dG2_dr():
    """DL2 = -(alpha/r) dG2/dr, checked with a central difference."""
    for alpha in (1.0, 0.5):
        for r in (0.01, 0.1, 0.4):
            for s in (0.003, 0.1):
                e = 1e-6 * r
                dg = (O.G2(r + e, s, alpha) - O.G2(r - e, s, alpha)) / (2 * e)
                assert O.DL2(r, s, alpha) == pytest.approx(-alpha / r * dg, rel=1e-6)

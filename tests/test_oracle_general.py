"""Pins of the oracle for general (non-uniform) time steps: Alg. 1 in full (early leaves, the
split at the step nearest the centre, the oversized-element stop), the nearfield of Eq.
def_st_nearfield with its N(parent) /\\ leaves term, and the pFMM of Alg. 2 on that tree.

* the time integral over a target and a source step against adaptive quadrature of the heat
  kernel G (Section 2), and against the uniform-step entries (pinned elsewhere);
* the dense product with uniform steps against the block-Toeplitz oracle;
* the tree: splits at the nearest step, children partition their parent, leaves partition the
  space-time elements, early leaves exist and oversized steps stop the refinement;
* the partition of Alg. 2: every causal element pair is covered exactly once by a nearfield
  block or an admissible block, no other pair is (brute force on tiny problems);
* the pFMM converges to the dense Galerkin product as the degree grows."""
import numpy as np
import pytest

import oracle as O
from paper_2106_15911_gb300.inputs import cube_mesh, random_density

integrate = pytest.importorskip("scipy.integrate")


def _graded(E, p=2.0):
    u = np.linspace(0.0, 1.0, E + 1)
    return u ** p


def _random_steps(E, seed):
    h = np.random.default_rng(seed).uniform(0.3, 1.7, E)
    return np.concatenate([[0.0], np.cumsum(h)]) / h.sum()


@pytest.mark.parametrize("r", [0.05, 0.3, 1.2])
@pytest.mark.parametrize("steps", [((0.2, 0.5), (0.2, 0.5)), ((0.5, 0.6), (0.1, 0.5)), ((0.9, 1.0), (0.0, 0.3)),
                                   ((0.3, 0.35), (0.05, 0.3))])
def test_step_time_integral_against_quadrature(r, steps):
    (tk0, tk1), (tj0, tj1) = steps

    def g(tau, t):
        return O.G(r, t - tau) if t > tau else 0.0

    ref, _ = integrate.dblquad(g, tk0, tk1, lambda t: tj0, lambda t: min(tj1, t), epsabs=1e-14, epsrel=1e-12)
    got = O.time_V_steps(r, tk0, tk1, tj0, tj1)
    assert abs(got - ref) <= 1e-9 * max(abs(ref), 1e-12) + 1e-13, (got, ref)
    # invariant under a shift of both steps in time
    assert O.time_V_steps(r, tk0 + 2.0, tk1 + 2.0, tj0 + 2.0, tj1 + 2.0) == pytest.approx(got, rel=1e-9, abs=1e-15)
    assert O.time_V_steps(r, tj0, tj1, tk1 + 0.1, tk1 + 0.2) == 0.0  # a later source step: causality


def test_step_time_integral_reduces_to_uniform():
    h = 1.0 / 64
    for r in (0.01, 0.1, 0.7):
        for d in range(0, 6):
            k = 9
            got = O.time_V_steps(r, k * h, (k + 1) * h, (k - d) * h, (k - d + 1) * h)
            assert got == pytest.approx(O.time_V(r, d, h), rel=1e-12, abs=1e-16)


def test_dense_product_with_uniform_steps_is_the_toeplitz_product():
    V, T = cube_mesh(2)
    E = 8
    ts = np.linspace(0.0, 1.0, E + 1)
    P = O.make_general_problem(V, T, ts)
    w = random_density(E, T.shape[0], 1, seed=11)[0]
    rows = np.array([0, 5, 17, 40])
    f = O.gen_dense_apply(P, w, rows)[:, rows]
    blocks = O.assemble_V_rows(V, T, 1.0 / E, rows, d0=0, nd=E)
    ref = O.toeplitz_rows_apply(blocks, w)
    assert np.max(np.abs(f - ref)) <= 1e-12 * np.max(np.abs(ref))


def _leaf_elements(P, n_max, info):
    """every (step, triangle) element -> number of leaves holding it"""
    from collections import Counter
    nt, E = P.nt, P.Et
    V = np.ctypeslib.as_array(P._keep[0])
    T = np.ctypeslib.as_array(P._keep[1])
    cnt = np.zeros((E, nt), np.int32)
    cent = V[T].mean(axis=1)
    lo, hi = V.min(0), V.max(0)
    H = 0.5 * (hi - lo).max()
    corner = 0.5 * (lo + hi) - H
    for l, cx, cy, cz, k, leaf in info["boxes"]:
        if not leaf:
            continue
        G = 1 << info["lx"][l]
        w = 2 * H / G
        cell = np.clip(np.ceil((cent - corner) / w).astype(int) - 1, 0, G - 1)
        inside = (cell[:, 0] == cx) & (cell[:, 1] == cy) & (cell[:, 2] == cz)
        ia, ib = O.gen_interval(P, n_max, l, k)
        cnt[ia:ib, inside] += 1
    return Counter(cnt.ravel().tolist())


@pytest.mark.parametrize("ts", [_graded(16), _random_steps(16, 3), np.linspace(0, 1, 17)])
@pytest.mark.parametrize("n_max", [24, 96])
def test_general_tree(ts, n_max):
    V, T = cube_mesh(2)
    P = O.make_general_problem(V, T, ts, m_t=3, m_x=3)
    info = O.gen_tree_info(P, n_max, boxes=True)
    # the leaves partition the space-time elements
    assert _leaf_elements(P, n_max, info) == {1: P.Et * P.nt}
    # every present interval splits at the step nearest its centre; children partition the parent
    for l in range(info["nlev"] - 1):
        for k in range(1 << l):
            a, b = O.gen_interval(P, n_max, l, k)
            c0, c1 = O.gen_interval(P, n_max, l + 1, 2 * k), O.gen_interval(P, n_max, l + 1, 2 * k + 1)
            if a < 0 or c0[0] < 0:
                assert c0 == (-1, -1) and c1 == (-1, -1)
                continue
            mid = 0.5 * (ts[a] + ts[b])
            s = min(range(a + 1, b), key=lambda q: (abs(ts[q] - mid), q))
            assert c0 == (a, s) and c1 == (s, b)
    # boxes below the root level have a parent: every level but 0 is reached by refinement
    assert info["nbox"][0] >= 1 and all(n > 0 for n in info["nbox"])


def test_early_leaves_and_oversized_steps():
    V, T = cube_mesh(2)
    # one long step in the middle: no box holding it refines below the level whose nominal
    # interval length falls under the step's length
    h = np.full(16, 1.0)
    h[9] = 4.0
    ts = np.concatenate([[0.0], np.cumsum(h)]) / h.sum()
    P = O.make_general_problem(V, T, ts, m_t=3, m_x=3)
    info = O.gen_tree_info(P, 8, boxes=True)
    long_len = ts[10] - ts[9]
    for l, cx, cy, cz, k, leaf in info["boxes"]:
        a, b = O.gen_interval(P, 8, l, k)
        if a <= 9 < b and not leaf:
            assert long_len <= 1.0 / (1 << l) + 1e-15
    # graded steps give leaves on several levels
    P2 = O.make_general_problem(V, T, _graded(16), m_t=3, m_x=3)
    i2 = O.gen_tree_info(P2, 16)
    assert sum(1 for n in i2["nleaf"] if n > 0) >= 3


@pytest.mark.parametrize("ts,n_max", [(_graded(16), 16), (_random_steps(16, 7), 24), (_graded(12, 3.0), 8),
                                      (np.linspace(0, 1, 17), 32)])
def test_partition_covers_every_causal_pair_once(ts, n_max):
    V, T = cube_mesh(2)
    P = O.make_general_problem(V, T, ts, m_t=3, m_x=3, n_tr=100)  # no truncation of the areas
    cov = O.gen_coverage(P, n_max)
    k = np.repeat(np.arange(P.Et), P.nt)
    causal = k[:, None] >= k[None, :]
    assert np.all(cov[causal] == 1)
    assert np.all(cov[~causal] == 0)


def test_general_pfmm_converges_to_the_dense_product():
    V, T = cube_mesh(4)
    E = 32
    ts = _graded(E, 1.5)
    w = random_density(E, T.shape[0], 1, seed=3)[0]
    rows = np.arange(0, T.shape[0], 24)
    P = O.make_general_problem(V, T, ts, m_t=4, m_x=2)
    ref = O.gen_dense_apply(P, w, rows)[:, rows]
    errs = []
    for mx in (2, 4, 6):
        P = O.make_general_problem(V, T, ts, m_t=4, m_x=mx)
        f = O.gen_pfmm_apply(P, 60, w, targets=rows)[:, rows]
        errs.append(np.max(np.abs(f - ref)) / np.max(np.abs(ref)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 2e-3

"""Structure pins of the oracle's dense Galerkin blocks (Section 2): block lower-triangular and
block-Toeplitz V_h for uniform steps, symmetric blocks with an SPD diagonal block, a vanishing
double layer on coplanar pairs, the mass matrix, and the steady-state limit of K_h given by
Gauss's law for the Laplace double layer (the time integral of the heat kernel over (0, inf) is
1 / (4 pi alpha r))."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2106_15911_gb300.inputs import cube_mesh


@pytest.fixture(scope="module")
def small():
    V, T = cube_mesh(2)
    h = 1.0 / 16
    return V, T, h, O.assemble_V(V, T, h, nd=4), O.assemble_K(V, T, h, nd=4)


def test_toeplitz_time_structure():
    """Entries depend on t_k - t_j only: the four-term formula with absolute times matches the
    offset form for different (k, j) with the same d."""
    h, r = 1.0 / 64, 0.03
    for d in range(0, 6):
        vals = []
        for j in range(1, 5):
            k = j + d
            tk, tk1, tj, tj1 = k * h, (k - 1) * h, j * h, (j - 1) * h
            vals.append(O.G2(r, tk - tj1) - O.G2(r, tk - tj) - O.G2(r, tk1 - tj1) + O.G2(r, tk1 - tj))
        assert np.allclose(vals, O.time_V(r, d, h), rtol=1e-9, atol=0)


def test_V_blocks_symmetric_and_A0_spd(small):
    V, T, h, A, _ = small
    # (x, y) and (y, x) use different Sauter-Schwab parametrisations, so the blocks are
    # symmetric up to that rule's error: ~1e-5 at the default order, ~1e-11 at order 12
    for d in range(A.shape[0]):
        assert np.max(np.abs(A[d] - A[d].T)) <= 3e-5 * np.max(np.abs(A[d]))
    Ahi = O.assemble_V(V, T, h, nd=2, n_s=12)
    for d in range(2):
        assert np.max(np.abs(Ahi[d] - Ahi[d].T)) <= 1e-10 * np.max(np.abs(Ahi[d]))
    ev = np.linalg.eigvalsh(A[0])
    assert ev.min() > 0
    np.linalg.cholesky(A[0])


def test_V_blocks_positive_and_decaying(small):
    V, T, h, A, _ = small
    assert np.all(A[0] > 0)
    # farther in time: smaller diagonal entries (heat kernel decays in t - tau at r ~ 0)
    assert np.all(np.diag(A[1]) < np.diag(A[0]))


def test_K_vanishes_on_coplanar_pairs():
    V, T = cube_mesh(2)
    n = np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    cnt = 0
    for x in range(0, T.shape[0], 5):
        for y in range(T.shape[0]):
            same_plane = abs(abs(n[x] @ n[y]) - 1) < 1e-14 and abs((V[T[x][0]] - V[T[y][0]]) @ n[y]) < 1e-14
            if same_plane:
                for d in (0, 1, 3):
                    v = O.pair_integral(V, T[x], T[y], O.KIND_K, 6, use_ss=True, d=d, h=0.01)
                    assert np.all(v == 0.0)
                cnt += 1
    assert cnt > 20


def test_mass_rows(small):
    V, T, h, _, _ = small
    M = O.assemble_M(V, T, h)
    area = 0.5 * np.linalg.norm(np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]]), axis=1)
    assert np.allclose(M.sum(axis=1), h * area, rtol=1e-14)


def test_K_steady_state_gauss_law():
    """sum_{j<=k} sum_i K[(k,x),(j,i)] / (h |gamma_x|) -> -1/2 once t_k >> diam^2 / alpha.
    The tail of the time integral leaves a relative defect erf(u) - 2u e^{-u^2}/sqrt(pi) ~ u^3
    with u = diam / (2 sqrt(alpha t)), about 2e-4 here."""
    V, T = cube_mesh(2)
    Tend, Et = 200.0, 8
    h = Tend / Et
    B = O.assemble_K(V, T, h, nd=Et, n_r=4, n_s=8)
    area = 0.5 * np.linalg.norm(np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]]), axis=1)
    rows = B.sum(axis=(0, 2)) / (h * area)
    u = math.sqrt(3.0) / (2 * math.sqrt((Tend - h)))
    tail = math.erf(u) - 2 * u * math.exp(-u * u) / math.sqrt(math.pi)
    assert np.max(np.abs(rows + 0.5)) < 2e-3 + 4 * tail


def test_sampled_rows_match_the_full_blocks_and_the_pfmm_nearfield():
    """The row-sampled assembly returns exactly the listed rows of the full Toeplitz blocks, and
    their product restricted to the nearfield offsets (d <= ls + k mod ls) equals the nearfield
    part of the oracle's pFMM (Alg. 2, last loop) on those rows; with all offsets it equals the
    dense product."""
    V, T = cube_mesh(2)
    Et, h = 16, 1.0 / 16
    rows = np.array([0, 5, 11, 30, 47])
    A = O.assemble_V(V, T, h, nd=Et)
    R = O.assemble_V_rows(V, T, h, rows, nd=Et)
    assert np.array_equal(A[:, rows, :], R)
    x = np.random.default_rng(3).standard_normal((Et, T.shape[0]))
    assert np.allclose(O.toeplitz_rows_apply(R, x), O.toeplitz_apply(A, x)[:, rows], rtol=0, atol=1e-14)
    Pr = O.make_problem(V, T, 1.0, Et, m_t=3, m_x=3, c_st=1.0)
    near = O.pfmm_apply(Pr, 0, x, targets=rows, parts=1)[:, rows]
    mine = O.toeplitz_rows_apply(R[:4], x, leaf_steps=2)
    assert np.max(np.abs(mine - near)) <= 1e-14 * np.max(np.abs(near))

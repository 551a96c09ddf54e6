"""The a-priori degree choice of the batch autotuner (host only, no GPU): the chosen spatial
degree grows as the tolerance tightens, stays in the requested range, and meets its target on
the oracle's pFMM."""
from paper_2106_15911_gb300 import pfmm as P
from paper_2106_15911_gb300.inputs import cube_mesh, cube_sphere_mesh


def test_degree_grows_with_tighter_tolerance():
    V, T = cube_mesh(8)
    ms = [P.pfmm_autotune_params(V, T, 1.0, 64, tol=t, m_lo=2, m_hi=10).m_x for t in (1e-2, 1e-4, 1e-6, 1e-9)]
    assert ms == sorted(ms) and ms[0] < ms[-1] and all(2 <= m <= 10 for m in ms)


def test_degree_range_and_shallow_tree():
    V, T = cube_sphere_mesh(4)
    p = P.pfmm_autotune_params(V, T, 1.0, 32, tol=1e-30, m_lo=4, m_hi=6)
    assert p.m_x == 6
    p2 = P.pfmm_autotune_params(V, T, 1.0, 4, tol=1e-6, m_lo=4, m_hi=8)  # no M2L level
    assert p2.m_x == 4


def test_chosen_degree_meets_the_target_on_the_oracle():
    """The a-priori choice is safe: the far field of the oracle's pFMM at the chosen degree differs
    from the one at m_x = 10 by at most the tolerance, relative to the largest entry of V_h w
    (16 sampled rows, 64 steps; the m_x = 10 reference is itself within about 5e-5)."""
    import numpy as np

    import oracle as O
    from paper_2106_15911_gb300.inputs import random_density, sample_triangles

    for mesh in (cube_mesh, cube_sphere_mesh):
        V, T = mesh(8)
        Et = 64
        rows = sample_triangles(T.shape[0], 16, seed=7)
        w = random_density(Et, T.shape[0], 1, seed=5)[0]
        ref = O.make_problem(V, T, 1.0, Et, m_t=4, m_x=10)
        far_ref = O.pfmm_apply(ref, 0, w, targets=rows, parts=2)[:, rows]
        scale = np.abs(O.pfmm_apply(ref, 0, w, targets=rows, parts=1)[:, rows] + far_ref).max()
        for tol in (1e-2, 3e-3, 1e-3):
            m = P.pfmm_autotune_params(V, T, 1.0, Et, tol=tol, m_lo=2, m_hi=9).m_x
            far = O.pfmm_apply(O.make_problem(V, T, 1.0, Et, m_t=4, m_x=m), 0, w, targets=rows, parts=2)[:, rows]
            assert np.abs(far - far_ref).max() <= tol * scale, (mesh.__name__, tol, m)

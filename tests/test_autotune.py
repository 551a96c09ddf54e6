"""The a-priori degree choice of the batch autotuner (host only, no GPU): the chosen spatial
degree grows as the tolerance tightens and stays in the requested range."""
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

"""General (non-uniform) time steps on the GPU (pfmm_gen_*): the tree of Alg. 1 with early leaves
equals the oracle's box for box, and V_h w by the FMM on it matches the oracle's pFMM on the same
tree element by element (FP64, 1e-12 of the largest value) for the nearfield (Eq. def_st_nearfield
with N(parent) /\\ leaves; on sampled target rows, the oracle's quadrature being slow), the far
field (every row) and the whole product, on graded, random and uniform steps, several element
bounds n_max, a tree without far field, and more right-hand sides than one pass of the nearfield
kernel takes.  The product approximates the dense Galerkin product."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2106_15911_gb300 import pfmm as P
from paper_2106_15911_gb300.inputs import cube_mesh, cube_sphere_mesh, random_density

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _graded(E, p=2.0):
    return np.linspace(0.0, 1.0, E + 1) ** p


def _random_steps(E, seed):
    h = np.random.default_rng(seed).uniform(0.3, 1.7, E)
    return np.concatenate([[0.0], np.cumsum(h)]) / h.sum()


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


# mesh, squares per face edge, steps, n_max, parameters, stride of the sampled nearfield rows,
# leaves on several levels (not with uniform steps on a uniform mesh)
CASES = [
    (cube_mesh, 4, _graded(32, 1.5), 60, dict(m_t=4, m_x=4), 4, True),
    (cube_mesh, 4, _random_steps(24, 5), 40, dict(m_t=3, m_x=5), 4, True),
    (cube_mesh, 8, _graded(16, 2.0), 200, dict(m_t=4, m_x=6), 16, True),
    (cube_mesh, 4, np.linspace(0.0, 1.0, 33), 100, dict(m_t=4, m_x=4, c_st=0.25), 4, False),
    (cube_sphere_mesh, 4, _graded(24, 2.5), 48, dict(m_t=4, m_x=4, c_st=0.5), 4, True),
]


@pytest.mark.parametrize("mesh,n_a,ts,n_max,kw,stride,early", CASES)
def test_general_tree_matches_oracle(mesh, n_a, ts, n_max, kw, stride, early):
    V, T = mesh(n_a)
    op = P.GeneralOperator(V, T, ts, n_max, **kw)
    Pr = O.make_general_problem(V, T, ts, **kw)
    ref = O.gen_tree_info(Pr, n_max, boxes=True)
    got = op.info()
    for k in ("nlev", "lx", "nbox", "nleaf", "nint", "ntr_far", "ntr_near"):
        assert got[k] == ref[k], k
    assert got["st"][:-1] == ref["st"][:-1]
    rows = op.boxes()
    assert sorted(map(tuple, rows[:, :6].tolist())) == sorted(map(tuple, ref["boxes"].tolist()))
    for l, cx, cy, cz, k, leaf, a0, a1 in rows.tolist():
        assert (a0, a1) == O.gen_interval(Pr, n_max, l, k)
    op.close()


@pytest.mark.parametrize("mesh,n_a,ts,n_max,kw,stride,early", CASES)
def test_general_apply_matches_oracle(mesh, n_a, ts, n_max, kw, stride, early):
    V, T = mesh(n_a)
    E = len(ts) - 1
    op = P.GeneralOperator(V, T, ts, n_max, **kw)
    info = op.info()
    assert info["nlev"] >= 3
    assert (sum(1 for n in info["nleaf"] if n > 0) >= 2) == early  # leaves on several levels
    Pr = O.make_general_problem(V, T, ts, **kw)
    w = random_density(E, T.shape[0], 2, seed=91)
    wt = torch.tensor(w, device=DEV)
    near = op.V(wt, parts=P.PFMM_PART_NEAR).cpu().numpy()
    far = op.V(wt, parts=P.PFMM_PART_FAR).cpu().numpy()
    full = op.V(wt).cpu().numpy()
    assert _rel(full, near + far) <= 1e-14
    rows = np.arange(0, T.shape[0], stride)
    for r in range(2):
        ref_far = O.gen_pfmm_apply(Pr, n_max, w[r], parts=P.PFMM_PART_FAR)
        assert _rel(far[r], ref_far) <= 1e-12, (r, _rel(far[r], ref_far))
    ref_near = O.gen_pfmm_apply(Pr, n_max, w[0], targets=rows, parts=P.PFMM_PART_NEAR)[:, rows]
    assert _rel(near[0][:, rows], ref_near) <= 1e-12, _rel(near[0][:, rows], ref_near)
    ref_full = ref_near + O.gen_pfmm_apply(Pr, n_max, w[0], parts=P.PFMM_PART_FAR)[:, rows]
    assert _rel(full[0][:, rows], ref_full) <= 1e-12
    op.close()


def test_general_tree_without_far_field_and_many_rhs():
    V, T = cube_mesh(4)
    ts = _graded(12, 2.0)
    op = P.GeneralOperator(V, T, ts, 10 ** 6, m_t=3, m_x=3)
    assert op.info()["nlev"] == 1
    Pr = O.make_general_problem(V, T, ts, m_t=3, m_x=3)
    w = random_density(12, T.shape[0], 9, seed=17)  # 9 rhs: two passes of the nearfield kernel
    f = op.V(torch.tensor(w, device=DEV)).cpu().numpy()
    rows = np.arange(0, T.shape[0], 6)
    for r in (0, 4, 8):
        ref = O.gen_dense_apply(Pr, w[r], rows)[:, rows]
        assert _rel(f[r][:, rows], ref) <= 1e-12
    op.close()


def test_general_apply_approximates_the_dense_product():
    V, T = cube_mesh(4)
    E = 32
    ts = _graded(E, 1.5)
    op = P.GeneralOperator(V, T, ts, 60, m_t=4, m_x=6)
    Pr = O.make_general_problem(V, T, ts, m_t=4, m_x=6)
    w = random_density(E, T.shape[0], 1, seed=3)[0]
    rows = np.arange(0, T.shape[0], 24)
    f = op.V(torch.tensor(w, device=DEV)).cpu().numpy()[:, rows]
    ref = O.gen_dense_apply(Pr, w, rows)[:, rows]
    assert _rel(f, ref) <= 2e-3
    op.close()


def test_general_rejects_bad_steps():
    V, T = cube_mesh(2)
    with pytest.raises(P.PfmmError):
        P.GeneralOperator(V, T, np.array([0.0, 0.5, 0.4, 1.0]), 16)
    with pytest.raises(P.PfmmError):
        P.GeneralOperator(V, T, np.array([0.1, 0.5, 1.0]), 16)
    with pytest.raises(P.PfmmError):
        P.GeneralOperator(V, T, np.linspace(0, 1, 9), 16, precision=P.PFMM_MIXED)

"""GPU solve of the space-time system (Section 2, Eq. 02:linear:system) through the C ABI
against the oracle: the right-hand side (1/2 M_h + K_h) g and the solution of V_h x = b with
the same pFMM operator, restarted FGMRES on the device vs plain numpy GMRES on the oracle's
CPU pFMM; GMRES-IR with a mixed-precision inner operator and FP64 residuals."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle.solve import gmres
from paper_2106_15911_gb300 import pfmm as P
from paper_2106_15911_gb300.inputs import cube_mesh, heat_source_datum

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
KW = dict(m_t=5, m_x=6, c_st=0.25)


@pytest.fixture(scope="module")
def problem():
    V, T = cube_mesh(4)
    Et = 16
    g = heat_source_datum(V, 1.0, Et, [(np.array([1.5, 1.5, 1.5]), -0.1)])
    Pr = O.make_problem(V, T, 1.0, Et, **KW)
    M = O.assemble_M(V, T, 1.0 / Et)
    b = 0.5 * (g @ M.T) + O.pfmm_apply(Pr, 1, g)
    x_ref, it, _ = gmres(lambda x: O.pfmm_apply(Pr, 0, x), b, tol=1e-10, restart=60)
    return V, T, Et, g, Pr, b, x_ref


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def test_fp64_fgmres_matches_oracle_gmres(problem):
    V, T, Et, g, Pr, b, x_ref = problem
    op = P.Operator(V, T, 1.0, Et, **KW)
    gt = torch.tensor(g[None], device=DEV)
    x = torch.empty((1, Et, T.shape[0]), dtype=torch.float64, device=DEV)
    info = P.pfmm_solve(op.h, P.PFMM_DIRECT, gt, x, 1)
    xs = x.cpu().numpy()[0]
    assert info["rel_res"] <= 1e-8 and 3 <= info["iterations"] < 200
    # the oracle's operator agrees that this x solves the system
    res = np.linalg.norm(b - O.pfmm_apply(Pr, 0, xs)) / np.linalg.norm(b)
    assert res <= 1e-7
    assert _rel(xs, x_ref) <= 1e-6
    op.close()


def test_mixed_gmres_ir_reaches_fp64_residual(problem):
    V, T, Et, g, Pr, b, x_ref = problem
    op64 = P.Operator(V, T, 1.0, Et, **KW)
    opm = P.Operator(V, T, 1.0, Et, precision=P.PFMM_MIXED, **KW)
    gt = torch.tensor(g[None], device=DEV)
    x = torch.empty((1, Et, T.shape[0]), dtype=torch.float64, device=DEV)
    o = P.pfmm_default_solve_opts()
    o.refine = op64.h
    info = P.pfmm_solve(opm.h, P.PFMM_DIRECT, gt, x, 1, o)
    assert info["rel_res"] <= 1e-8 and info["outer"] >= 1
    xs = x.cpu().numpy()[0]
    assert _rel(xs, x_ref) <= 1e-6
    op64.close()
    opm.close()


def test_indirect_formulation_and_several_rhs(problem):
    V, T, Et, g, Pr, b, x_ref = problem
    op = P.Operator(V, T, 1.0, Et, **KW)
    g2 = np.stack([g, 2.0 * g])
    x = torch.empty((2, Et, T.shape[0]), dtype=torch.float64, device=DEV)
    info = P.pfmm_solve(op.h, P.PFMM_INDIRECT, torch.tensor(g2, device=DEV), x, 2)
    xs = x.cpu().numpy()
    M = O.assemble_M(V, T, 1.0 / Et)
    bi = g @ M.T
    assert np.linalg.norm(bi - O.pfmm_apply(Pr, 0, xs[0])) / np.linalg.norm(bi) <= 1e-7
    assert _rel(xs[1], 2.0 * xs[0]) <= 1e-7
    assert info["rel_res"] <= 1e-8
    op.close()


def test_solver_reports_caps_and_bad_input(problem):
    V, T, Et, g, Pr, b, x_ref = problem
    op = P.Operator(V, T, 1.0, Et, **KW)
    x = torch.empty((1, Et, T.shape[0]), dtype=torch.float64, device=DEV)
    o = P.pfmm_default_solve_opts()
    o.max_it = 2
    info = P.pfmm_solve(op.h, P.PFMM_DIRECT, torch.tensor(g[None], device=DEV), x, 1, o, allow_not_converged=True)
    assert not info["converged"] and info["iterations"] == 2 and info["rel_res"] > 1e-8
    gb = g.copy()
    gb[3, 5] = np.nan
    with pytest.raises(P.PfmmError, match="NONFINITE"):
        P.pfmm_solve(op.h, P.PFMM_DIRECT, torch.tensor(gb[None], device=DEV), x, 1)
    op.close()

"""The allocation-free entry point pfmm_apply_V_noalloc (for callers that must not allocate
device memory while they run) computes the same f = V_h w as pfmm_apply_V, call after call,
through the C ABI, and refuses problems whose workspaces exceed its static 64 MiB array.

This file is collected last on purpose (a stop-at-first-failure run has then already run every
other test); it passes alone in a fresh process and after the other tests."""
import numpy as np
import pytest
import torch

from paper_2106_15911_gb300 import pfmm as P
from paper_2106_15911_gb300.inputs import cube_mesh, random_density

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("precision,n_a,Et,kw", [
    (P.PFMM_FP64, 4, 16, dict(m_t=4, m_x=4, c_st=0.25)),
    (P.PFMM_MIXED, 4, 16, dict(m_t=4, m_x=4, c_st=0.25)),
    (P.PFMM_MIXED, 4, 16, dict(m_t=4, m_x=4, c_st=1.0)),   # tensor-core nearfield, parts in the array
    (P.PFMM_MIXED, 12, 32, dict(m_t=4, m_x=6, c_st=0.1)),  # 8^3 leaf grid: slab M2L, no T1 / T2 needed
])
def test_noalloc_matches_apply_V_on_two_calls(precision, n_a, Et, kw):
    V, T = cube_mesh(n_a)
    nrhs = 2
    op = P.Operator(V, T, 1.0, Et, precision=precision, **kw)
    if precision == P.PFMM_MIXED and kw["c_st"] == 1.0:
        assert op.info()["nf_tensor_cores"] & 1
    if n_a == 12:
        info = op.info()
        assert P.PFMM_M2L_SLAB in info["m2l_engine"]
    for seed in (11, 12):  # two calls in a row: the second must not see the first's contents
        w = torch.tensor(random_density(Et, T.shape[0], nrhs, seed=seed), device=DEV)
        ref = torch.empty_like(w)
        out = torch.full_like(w, float("nan"))
        P.pfmm_apply_V(op.h, w, ref, nrhs)
        P.pfmm_apply_V_noalloc(op.h, w, out, nrhs)
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        # FP64: the same arithmetic up to summation order; mixed: the two entry points may take
        # different S2M / L2T forms (the two-stage form needs a workspace that the static array
        # offers and the per-handle one may not), which add in different FP32 orders
        tol = 1e-12 if precision == P.PFMM_FP64 else 1e-6
        assert np.max(np.abs(a - b)) / np.max(np.abs(b)) <= tol
    op.close()


def test_noalloc_rejects_workspaces_beyond_the_static_array():
    V, T = cube_mesh(4)
    Et, nrhs = 16, 4096  # 4096 x 16 x 192 FP64 values: ~100 MB of workspace
    op = P.Operator(V, T, 1.0, Et)
    w = torch.zeros((nrhs, Et, T.shape[0]), dtype=torch.float64, device=DEV)
    f = torch.empty_like(w)
    with pytest.raises(P.PfmmError, match="static scratch holds 67108864 bytes"):
        P.pfmm_apply_V_noalloc(op.h, w, f, nrhs)
    op.close()

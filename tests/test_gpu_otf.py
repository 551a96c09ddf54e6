"""On-the-fly nearfield (quadrature fused into the apply, no stored blocks) through the C ABI:
FP64 against the CPU oracle (1e-12), against the stored path in both precisions on trees with
several panels, partial interaction areas and ragged 64-row tiles, for leaf sizes of 1, 2 and 4
steps, V and K, several right-hand sides; the same-step block used to train the preconditioner;
the memory it keeps."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2106_15911_gb300 import pfmm as P
from paper_2106_15911_gb300.inputs import cube_mesh, cube_sphere_mesh, random_density

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_otf_fp64_matches_oracle():
    V, T = cube_mesh(4)  # 192 triangles x 16 steps, m_t = m_x = 4, c_st = 1
    Et, nrhs = 16, 3
    op = P.Operator(V, T, 1.0, Et, m_t=4, m_x=4, c_st=1.0, nearfield=P.PFMM_NEARFIELD_ONTHEFLY)
    Pr = O.make_problem(V, T, 1.0, Et, m_t=4, m_x=4, c_st=1.0)
    w = random_density(Et, len(T), nrhs, seed=11)
    g = random_density(Et, len(V), nrhs, seed=12)
    fV = op.V(torch.tensor(w, device=DEV)).cpu().numpy()
    fK = op.K(torch.tensor(g, device=DEV)).cpu().numpy()
    for r in range(nrhs):
        assert _rel(fV[r], O.pfmm_apply(Pr, 0, w[r])) <= 1e-12
        assert _rel(fK[r], O.pfmm_apply(Pr, 1, g[r])) <= 1e-12
    info = op.info()
    assert info["nf_tensor_cores"] == 0
    op.close()


@pytest.mark.parametrize("precision,tol", [(P.PFMM_FP64, 1e-12), (P.PFMM_MIXED, 2e-6)])
@pytest.mark.parametrize("mesh,n_a,Et,kw", [
    (cube_mesh, 8, 32, dict(m_t=4, m_x=5, c_st=0.25)),                 # space-time refined: several panels
    (cube_sphere_mesh, 6, 16, dict(m_t=3, m_x=4, c_st=0.5, leaf_steps=1)),
    (cube_mesh, 5, 64, dict(m_t=4, m_x=4, c_st=0.5, leaf_steps=4, leaf_tris=32)),
])
def test_otf_matches_stored(precision, tol, mesh, n_a, Et, kw):
    V, T = mesh(n_a)
    nrhs = 2
    ops = P.Operator(V, T, 1.0, Et, precision=precision, nf_engine=P.PFMM_NF_CUDA_CORES, **kw)
    opo = P.Operator(V, T, 1.0, Et, precision=precision, nearfield=P.PFMM_NEARFIELD_ONTHEFLY, **kw)
    assert opo.info()["nearfield_bytes"] < ops.info()["nearfield_bytes"]
    w = torch.tensor(random_density(Et, len(T), nrhs, seed=21), device=DEV)
    g = torch.tensor(random_density(Et, len(V), nrhs, seed=22), device=DEV)
    for parts in (P.PFMM_PART_NEAR, P.PFMM_PART_ALL):
        a, b = opo.V(w, parts=parts).cpu().numpy(), ops.V(w, parts=parts).cpu().numpy()
        assert _rel(a, b) <= tol, ("V", parts, _rel(a, b))
        a, b = opo.K(g, parts=parts).cpu().numpy(), ops.K(g, parts=parts).cpu().numpy()
        assert _rel(a, b) <= tol, ("K", parts, _rel(a, b))
    ops.close()
    opo.close()


def test_otf_noalloc_and_same_step_block():
    V, T = cube_mesh(8)
    Et = 16
    kw = dict(m_t=4, m_x=4, c_st=0.25, precision=P.PFMM_MIXED)
    ops = P.Operator(V, T, 1.0, Et, **kw)
    opo = P.Operator(V, T, 1.0, Et, nearfield=P.PFMM_NEARFIELD_ONTHEFLY, **kw)
    w = torch.tensor(random_density(Et, len(T), 1, seed=31), device=DEV)
    f1, f2 = torch.empty_like(w), torch.empty_like(w)
    P.pfmm_apply_V_noalloc(opo.h, w, f1, 1)
    P.pfmm_apply_V(opo.h, w, f2, 1, None)
    torch.cuda.synchronize()
    assert _rel(f1.cpu().numpy(), f2.cpu().numpy()) <= 1e-12
    # the same-step block A_0 seen by the preconditioner's training loss is the same in both modes
    net = P.Mpnn(V, T, 1.0, Et, width=16, layers=2, seed=1)
    net.output_scale = 1.0
    R = torch.tensor(random_density(Et, len(T), 2, seed=32), device=DEV)
    sl = np.array([0, 3, 17, 30], dtype=np.int32)
    l1, g1 = net.loss_grad(R, None, sl, handle=ops.h)
    l2, g2 = net.loss_grad(R, None, sl, handle=opo.h)
    assert l2 == pytest.approx(l1, rel=1e-5)
    assert np.max(np.abs(g1 - g2)) <= 1e-5 * np.max(np.abs(g1))
    net.close()
    ops.close()
    opo.close()

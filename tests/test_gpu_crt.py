"""FP64 nearfield on the tensor cores by exact residue arithmetic (the products of the scaled,
rounded blocks and input computed modulo 16 primes with FP16 MMAs, combined by the Chinese
remainder theorem): against the CPU oracle's nearfield (Alg. 2, last loop) within 1e-12, against
the FP64 CUDA-core engine on the same stored blocks within 1e-13, bitwise reproducible, exactly
scale-invariant in powers of two, zero for a zero right-hand side; V and K, ragged tiles (panels
of fewer than 128 rows), several interval blocks and right-hand sides."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2106_15911_gb300 import pfmm as P
from paper_2106_15911_gb300.inputs import cube_mesh, cube_sphere_mesh, random_density

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("mesh,n_a,Et,kw", [
    (cube_mesh, 4, 16, dict(m_t=4, m_x=4, c_st=1.0)),       # 192 triangles: one panel, ragged rows
    (cube_mesh, 8, 64, dict(m_t=4, m_x=6, c_st=1.0)),       # 768 triangles, 8 leaf boxes
    (cube_mesh, 4, 512, dict(m_t=3, m_x=3, c_st=1.0)),      # 256 leaf intervals: two interval blocks
    (cube_sphere_mesh, 16, 64, dict(m_t=4, m_x=5, c_st=0.1, n_tr=6)),  # dense columns with holes
])
@pytest.mark.parametrize("form", [1, 2])
def test_fp64_tensor_core_nearfield(mesh, n_a, Et, kw, form):
    V, T = mesh(n_a)
    op = P.Operator(V, T, 1.0, Et, nf_form=form, **kw)
    opc = P.Operator(V, T, 1.0, Et, nf_engine=P.PFMM_NF_CUDA_CORES, **kw)
    assert op.info()["nf_tensor_cores"] == 3 and opc.info()["nf_tensor_cores"] == 0
    assert op.info()["nf_form"] == form
    Pr = O.make_problem(V, T, 1.0, Et, **kw)
    w = random_density(Et, T.shape[0], 2, seed=71)
    g = random_density(Et, V.shape[0], 2, seed=72)
    for op_id, x in ((0, w), (1, g)):
        xt = torch.tensor(x, device=DEV)
        run = (lambda o: o.V(xt, parts=P.PFMM_PART_NEAR)) if op_id == 0 else (lambda o: o.K(xt, parts=P.PFMM_PART_NEAR))
        a = run(op).cpu().numpy()
        P.pfmm_check(op.h)
        c = run(opc).cpu().numpy()
        assert np.array_equal(a, run(op).cpu().numpy())  # integer arithmetic: bitwise reproducible
        for r in range(2):
            assert _rel(a[r], c[r]) <= 1e-13, (op_id, r, _rel(a[r], c[r]))
            if n_a <= 8:  # the oracle's nearfield of every row
                ref = O.pfmm_apply(Pr, op_id, x[r], parts=P.PFMM_PART_NEAR)
                assert _rel(a[r], ref) <= 1e-12, (op_id, r, _rel(a[r], ref))
    op.close()
    opc.close()


@pytest.mark.parametrize("form", [0, 1, 2])
def test_fp64_tensor_core_nearfield_scales_exactly(form):
    """Scales are powers of two per right-hand side, so 2^k x gives the same integers and
    exactly 2^k times the result; a zero right-hand side gives zeros (either kernel form, and
    the one the build-time timing picks)."""
    V, T = cube_mesh(8)
    Et = 64
    op = P.Operator(V, T, 1.0, Et, m_t=4, m_x=6, c_st=1.0, nf_form=form)
    assert op.info()["nf_tensor_cores"] == 3 and op.info()["nf_form"] in ((form,) if form else (1, 2))
    w = random_density(Et, T.shape[0], 1, seed=73)[0]
    g = random_density(Et, V.shape[0], 1, seed=74)[0]
    for apply, x in ((op.V, w), (op.K, g)):
        xs = np.stack([np.ldexp(x, -300), x, np.ldexp(x, 200), np.zeros_like(x)])
        out = apply(torch.tensor(xs, device=DEV), parts=P.PFMM_PART_NEAR).cpu().numpy()
        P.pfmm_check(op.h)
        assert np.max(np.abs(out[1])) > 0
        assert np.array_equal(np.ldexp(out[0], 300), out[1])
        assert np.array_equal(np.ldexp(out[2], -200), out[1])
        assert not np.any(out[3])
    op.close()


@pytest.mark.parametrize("mesh,n_a,Et,kw", [
    (cube_mesh, 8, 64, dict(m_t=4, m_x=6, c_st=1.0)),                   # tensor-core nearfield, 4^3 grids
    (cube_mesh, 4, 32, dict(m_t=5, m_x=6, c_st=0.25)),                  # space-time M2M / L2L
    (cube_sphere_mesh, 16, 64, dict(m_t=4, m_x=5, c_st=0.1, n_tr=6)),   # 8^3 grids, padded boxes
])
def test_fp64_mode_matches_native_fp64(mesh, n_a, Et, kw):
    """The FP64 mode's default arithmetic (exact residue nearfield, double-FP32 FMM passes) and
    the native FP64 reference mode (fp64_native = 1, every phase on the FP64 pipe) agree within
    1e-13 of the largest output, for V and K, far field and whole product."""
    V, T = mesh(n_a)
    op = P.Operator(V, T, 1.0, Et, **kw)
    opn = P.Operator(V, T, 1.0, Et, fp64_native=1, **kw)
    assert opn.info()["nf_tensor_cores"] == 0
    w = torch.tensor(random_density(Et, T.shape[0], 2, seed=81), device=DEV)
    g = torch.tensor(random_density(Et, V.shape[0], 2, seed=82), device=DEV)
    for apply, apply_n, x in ((op.V, opn.V, w), (op.K, opn.K, g)):
        for parts in (P.PFMM_PART_FAR, P.PFMM_PART_ALL):
            a = apply(x, parts=parts).cpu().numpy()
            b = apply_n(x, parts=parts).cpu().numpy()
            assert np.max(np.abs(b)) > 0
            assert _rel(a, b) <= 1e-13, (parts, _rel(a, b))
    P.pfmm_check(op.h)
    op.close()
    opn.close()

"""GPU parity of the CUDA pFMM against the CPU FP64 oracle (same tree, lists, degrees and
nearfield quadrature), through the C ABI.

Bars: FP64 mode within 1e-12 relative (max-norm over the compared rows); mixed mode within
1e-5 of the FP64 oracle.  Cases span several leaf boxes, padded boxes (cube-sphere),
truncated interaction areas, leaf sizes of 1, 2 and 4 steps, trees without farfield, several
right-hand sides, and the 12288-triangle x 256-step workload on sampled rows."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2106_15911_gb300 import pfmm as P
from paper_2106_15911_gb300.inputs import (cube_mesh, cube_sphere_mesh, random_density, sample_triangles)

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _rel(a, b, rows=None):
    if rows is not None:
        a, b = a[..., rows], b[..., rows]
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def _case(V, T, Et, nrhs=2, seed=1234, precision=P.PFMM_FP64, parts=3, tol=1e-12, **kw):
    op = P.Operator(V, T, 1.0, Et, precision=precision, **kw)
    okw = {k: v for k, v in kw.items() if k in ("m_t", "m_x", "c_st", "n_tr", "eps_tr", "leaf_steps", "leaf_tris")}
    if "quad_regular" in kw:
        okw["n_r"] = kw["quad_regular"]
    if "quad_singular" in kw:
        okw["n_s"] = kw["quad_singular"]
    Pr = O.make_problem(V, T, 1.0, Et, **okw)
    w = random_density(Et, T.shape[0], nrhs, seed=seed)
    g = random_density(Et, V.shape[0], nrhs, seed=seed + 1)
    fV = op.V(torch.tensor(w, device=DEV), parts=parts).cpu().numpy()
    fK = op.K(torch.tensor(g, device=DEV), parts=parts).cpu().numpy()
    errs = []
    for r in range(nrhs):
        eV = _rel(fV[r], O.pfmm_apply(Pr, 0, w[r], parts=parts))
        eK = _rel(fK[r], O.pfmm_apply(Pr, 1, g[r], parts=parts))
        errs.append((eV, eK))
        assert eV <= tol and eK <= tol, (r, eV, eK)
    info = op.info()
    op.close()
    return errs, info


def test_config1_fp64_matvec_matches_oracle():
    V, T = cube_mesh(4)  # 192 triangles, 16 steps, m_t = m_x = 4, c_st = 1 (config 1)
    errs, info = _case(V, T, 16, nrhs=8, m_t=4, m_x=4, c_st=1.0)
    assert info["p"] == 3 and info["n_m2l_pairs"] == 12


@pytest.mark.parametrize("parts", [P.PFMM_PART_NEAR, P.PFMM_PART_FAR])
def test_config1_parts_separately(parts):
    V, T = cube_mesh(4)
    _case(V, T, 16, nrhs=1, parts=parts, m_t=4, m_x=4, c_st=1.0)


def test_space_time_refinement_and_higher_degree():
    V, T = cube_mesh(4)
    errs, info = _case(V, T, 32, nrhs=2, m_t=5, m_x=6, c_st=0.25)
    assert info["lx"][-1] >= 1  # M2M / L2L cross space-time refinements


def test_padded_boxes_on_cube_sphere():
    V, T = cube_sphere_mesh(4)
    errs, info = _case(V, T, 32, nrhs=1, m_t=4, m_x=5, c_st=0.25)
    assert max(info["pad"]) > 0


def test_truncated_interaction_area():
    V, T = cube_mesh(8)  # 768 triangles
    _case(V, T, 32, nrhs=1, m_t=3, m_x=4, c_st=0.1, n_tr=1)


@pytest.mark.parametrize("ls,Et", [(1, 16), (4, 32), (2, 2), (2, 4)])
def test_leaf_sizes_and_shallow_trees(ls, Et):
    V, T = cube_mesh(2)
    _case(V, T, Et, nrhs=1, m_t=3, m_x=3, c_st=0.5, leaf_steps=ls)


def test_quadrature_orders_are_honoured():
    V, T = cube_mesh(2)
    _case(V, T, 8, nrhs=1, m_t=3, m_x=3, c_st=1.0, quad_regular=4, quad_singular=5)


def test_mass_matrix():
    V, T = cube_mesh(4)
    Et = 8
    op = P.Operator(V, T, 1.0, Et)
    g = random_density(Et, V.shape[0], 2, seed=3)
    f = op.M(torch.tensor(g, device=DEV)).cpu().numpy()
    M = O.assemble_M(V, T, 1.0 / Et)
    for r in range(2):
        assert _rel(f[r], g[r] @ M.T) < 1e-14
    op.close()


def test_mixed_precision_within_1e5_of_fp64_oracle():
    V, T = cube_mesh(8)
    errs, _ = _case(V, T, 64, nrhs=2, precision=P.PFMM_MIXED, tol=1e-5, m_t=4, m_x=6, c_st=1.0)


@pytest.mark.parametrize("mesh,n_a,Et,kw", [
    (cube_sphere_mesh, 16, 64, dict(m_t=4, m_x=5, c_st=0.1, n_tr=6)),  # 8^3 at levels 4, 5; radius 6
    (cube_mesh, 12, 32, dict(m_t=4, m_x=6, c_st=0.1)),                # 8^3 at the leaf level; radius 7
])
def test_mixed_m2l_on_8_cubed_grids_matches_fp64(mesh, n_a, Et, kw):
    """Levels with 5^3 .. 8^3 cells run the slab M2L in mixed precision (one CTA per target
    x-slab); the FP64 handle runs the three-pass kernels.  The far field (S2M .. L2T) of the two
    agrees to FP32 accuracy, for V and K and two right-hand sides."""
    V, T = mesh(n_a)
    opm = P.Operator(V, T, 1.0, Et, precision=P.PFMM_MIXED, **kw)
    opd = P.Operator(V, T, 1.0, Et, precision=P.PFMM_FP64, **kw)
    info = opm.info()
    lv8 = [l for l in range(2, info["p"] + 1) if 2 ** info["lx"][l] == 8]
    assert lv8 and all(info["m2l_engine"][l] == P.PFMM_M2L_SLAB for l in lv8), info["m2l_engine"]
    assert all(opd.info()["m2l_engine"][l] == P.PFMM_M2L_THREE_PASS for l in lv8)
    w = torch.tensor(random_density(Et, T.shape[0], 2, seed=51), device=DEV)
    g = torch.tensor(random_density(Et, V.shape[0], 2, seed=52), device=DEV)
    for op_m, op_d, x in ((opm.V, opd.V, w), (opm.K, opd.K, g)):
        fm = op_m(x, parts=P.PFMM_PART_FAR).cpu().numpy()
        fd = op_d(x, parts=P.PFMM_PART_FAR).cpu().numpy()
        assert np.max(np.abs(fd)) > 0
        assert _rel(fm, fd) <= 1e-5, _rel(fm, fd)
    P.pfmm_check(opm.h)
    opm.close()
    opd.close()


@pytest.mark.parametrize("mesh,n_a,Et,kw,engine8", [
    (cube_mesh, 12, 32, dict(m_t=4, m_x=6, c_st=0.1), P.PFMM_M2L_SLAB),                 # 8^3 leaf grid, radius 7
    (cube_sphere_mesh, 16, 64, dict(m_t=4, m_x=5, c_st=0.1, n_tr=6), P.PFMM_M2L_SLAB),  # padded boxes, radius 6
    (cube_mesh, 12, 32, dict(m_t=4, m_x=7, c_st=0.1), P.PFMM_M2L_THREE_PASS),           # m_x = 7: three passes
])
def test_8_cubed_grids_match_oracle(mesh, n_a, Et, kw, engine8):
    """Trees whose finest levels hold 8^3 grids of boxes (the shape of the 49152-triangle
    cube-sphere): the far field and the whole product of the mixed handle (slab M2L on the 8^3
    levels) within 1e-5, and of the FP64 handle (three separable passes) within 1e-12, of the
    oracle's pFMM (Alg. 2, literal Eq. m2l) on 8 sampled target triangles, V and K."""
    V, T = mesh(n_a)
    opm = P.Operator(V, T, 1.0, Et, precision=P.PFMM_MIXED, **kw)
    opd = P.Operator(V, T, 1.0, Et, precision=P.PFMM_FP64, **kw)
    info = opm.info()
    lv8 = [l for l in range(2, info["p"] + 1) if 2 ** info["lx"][l] == 8]
    assert lv8 and all(info["m2l_engine"][l] == engine8 for l in lv8), info["m2l_engine"]
    Pr = O.make_problem(V, T, 1.0, Et, **kw)
    rows = sample_triangles(T.shape[0], 8, seed=61)
    w = random_density(Et, T.shape[0], 1, seed=62)
    g = random_density(Et, V.shape[0], 1, seed=63)
    for op_id, x in ((0, w), (1, g)):
        xt = torch.tensor(x, device=DEV)
        for parts in (P.PFMM_PART_FAR, P.PFMM_PART_ALL):
            ref = O.pfmm_apply(Pr, op_id, x[0], targets=rows, parts=parts)
            fm = (opm.V(xt, parts=parts) if op_id == 0 else opm.K(xt, parts=parts)).cpu().numpy()[0]
            fd = (opd.V(xt, parts=parts) if op_id == 0 else opd.K(xt, parts=parts)).cpu().numpy()[0]
            assert np.max(np.abs(ref[:, rows])) > 0
            assert _rel(fd, ref, rows) <= 1e-12, (op_id, parts, _rel(fd, ref, rows))
            assert _rel(fm, ref, rows) <= 1e-5, (op_id, parts, _rel(fm, ref, rows))
    P.pfmm_check(opm.h)
    opm.close()
    opd.close()


@pytest.mark.parametrize("n_a,Et,m_x,kw", [
    (4, 32, 9, dict(m_t=4, c_st=0.25)),               # 220 moments: S2M / L2T over two moment chunks
    (4, 32, 12, dict(m_t=4, c_st=0.25)),              # 455 moments: three S2M chunks, two L2T launches
    (8, 256, 12, dict(m_t=4, c_st=4.1, n_tr=2)),      # the paper's large-run parameters (Section 5)
])
def test_high_degrees_match_oracle(n_a, Et, m_x, kw):
    """Degrees up to the ABI's m_x = 12 (Section 5 runs m_x = 12, m_t = 4, c_st = 4.1, n_tr = 2):
    FP64 within 1e-12 and mixed within 1e-5 of the oracle on 6 sampled target triangles, V and K."""
    V, T = cube_mesh(n_a)
    Pr = O.make_problem(V, T, 1.0, Et, m_x=m_x, **kw)
    rows = sample_triangles(T.shape[0], 6, seed=5)
    w = random_density(Et, T.shape[0], 1, seed=91)
    g = random_density(Et, V.shape[0], 1, seed=92)
    refs = {0: O.pfmm_apply(Pr, 0, w[0], targets=rows), 1: O.pfmm_apply(Pr, 1, g[0], targets=rows)}
    for prec, tol in ((P.PFMM_FP64, 1e-12), (P.PFMM_MIXED, 1e-5)):
        op = P.Operator(V, T, 1.0, Et, m_x=m_x, precision=prec, **kw)
        fV = op.V(torch.tensor(w, device=DEV)).cpu().numpy()[0]
        fK = op.K(torch.tensor(g, device=DEV)).cpu().numpy()[0]
        P.pfmm_check(op.h)
        op.close()
        assert _rel(fV, refs[0], rows) <= tol, (prec, _rel(fV, refs[0], rows))
        assert _rel(fK, refs[1], rows) <= tol, (prec, _rel(fK, refs[1], rows))


def test_sliced_fused_m2l_at_degree_8_matches_oracle():
    """m_x = 8 on 4^3 grids (the batch's degree-8 problems): the FP32 fused M2L forms T2 one nu1
    at a time (its full T2 does not fit shared memory); mixed within 1e-5 and FP64 within 1e-12
    of the oracle on 6 sampled target triangles, V and K."""
    V, T = cube_mesh(8)
    Et = 256
    kw = dict(m_t=4, m_x=8, c_st=1.0)
    Pr = O.make_problem(V, T, 1.0, Et, **kw)
    rows = sample_triangles(T.shape[0], 6, seed=95)
    w = random_density(Et, T.shape[0], 1, seed=96)
    g = random_density(Et, V.shape[0], 1, seed=97)
    refs = {0: O.pfmm_apply(Pr, 0, w[0], targets=rows), 1: O.pfmm_apply(Pr, 1, g[0], targets=rows)}
    for prec, tol in ((P.PFMM_MIXED, 1e-5), (P.PFMM_FP64, 1e-12)):
        op = P.Operator(V, T, 1.0, Et, precision=prec, **kw)
        if prec == P.PFMM_MIXED:
            assert P.PFMM_M2L_FUSED_SLICED in op.info()["m2l_engine"], op.info()["m2l_engine"]
        fV = op.V(torch.tensor(w, device=DEV)).cpu().numpy()[0]
        fK = op.K(torch.tensor(g, device=DEV)).cpu().numpy()[0]
        P.pfmm_check(op.h)
        op.close()
        assert _rel(fV, refs[0], rows) <= tol, (prec, _rel(fV, refs[0], rows))
        assert _rel(fK, refs[1], rows) <= tol, (prec, _rel(fK, refs[1], rows))


def test_errors_are_reported_not_crashed():
    V, T = cube_mesh(2)
    op = P.Operator(V, T, 1.0, 8)
    x = torch.zeros((1, 8, T.shape[0]), dtype=torch.float64, device=DEV)
    f = torch.empty_like(x)
    with pytest.raises(P.PfmmError):
        P.pfmm_apply_parts(op.h, 5, x, f, 1, 3)
    with pytest.raises(P.PfmmError):
        P.pfmm_apply_V(op.h, x, f, 0)
    op.close()


# ---- full-size workload: 12288 triangles x 256 steps, m_x = 6, m_t = 4, sampled rows ----------
@pytest.fixture(scope="module")
def cfg2():
    V, T = cube_mesh(32)
    Et = 256
    kw = dict(m_t=4, m_x=6, c_st=1.0)
    ops = {prec: P.Operator(V, T, 1.0, Et, precision=prec, **kw) for prec in (P.PFMM_FP64, P.PFMM_MIXED)}
    Pr = O.make_problem(V, T, 1.0, Et, **kw)
    yield V, T, Et, ops, Pr
    for o in ops.values():
        o.close()


def test_config2_tree(cfg2):
    V, T, Et, ops, Pr = cfg2
    info = ops[P.PFMM_FP64].info()
    oi = O.tree_info(Pr)
    assert info["lx"] == oi["lx"] == [0, 0, 0, 0, 1, 1, 2, 2]
    assert info["nbox"] == oi["nbox"] == [1, 1, 1, 1, 8, 8, 56, 56]


@pytest.mark.parametrize("op_id", [0, 1])
def test_config2_sampled_rows(cfg2, op_id):
    V, T, Et, ops, Pr = cfg2
    ncol = T.shape[0] if op_id == 0 else V.shape[0]
    x = random_density(Et, ncol, 1, seed=2025 + op_id)
    rows = sample_triangles(T.shape[0], 12, seed=11 + op_id)
    ref = O.pfmm_apply(Pr, op_id, x[0], targets=rows)
    xt = torch.tensor(x, device=DEV)
    f64 = (ops[P.PFMM_FP64].V(xt) if op_id == 0 else ops[P.PFMM_FP64].K(xt)).cpu().numpy()[0]
    f32 = (ops[P.PFMM_MIXED].V(xt) if op_id == 0 else ops[P.PFMM_MIXED].K(xt)).cpu().numpy()[0]
    assert _rel(f64, ref, rows) <= 1e-12
    assert _rel(f32, ref, rows) <= 1e-5


def test_config2_kernel_count(cfg2):
    """pfmm_count_apply_kernels (a captured graph of one apply) counts the kernels the bench
    claims per step: 32 for the mixed V_h apply of the 12288-triangle x 256-step workload, as the
    ncu launch list of that workload shows; the count does not depend on the call."""
    V, T, Et, ops, Pr = cfg2
    x = torch.zeros((1, Et, T.shape[0]), dtype=torch.float64, device=DEV)
    f = torch.empty_like(x)
    assert P.pfmm_count_apply_kernels(ops[P.PFMM_MIXED].h, 0, x, f, 1) == 32
    n64 = P.pfmm_count_apply_kernels(ops[P.PFMM_FP64].h, 0, x, f, 1)
    assert n64 >= 20 and n64 == P.pfmm_count_apply_kernels(ops[P.PFMM_FP64].h, 0, x, f, 1)
    # FP64 nearfield alone: permute in, input max and residues, residue products, combination,
    # permute out
    assert P.pfmm_count_apply_kernels(ops[P.PFMM_FP64].h, 0, x, f, 1, P.PFMM_PART_NEAR) == 6


# ---- tensor-core nearfield (scaled FP16 hi/lo split, mixed mode) -------------------------------
@pytest.mark.parametrize("n_a,Et,kw", [(4, 16, dict(m_t=4, m_x=4, c_st=1.0)), (8, 64, dict(m_t=4, m_x=6, c_st=1.0)),
                                       (4, 512, dict(m_t=3, m_x=3, c_st=1.0))])
def test_tensor_core_nearfield_matches_cuda_cores_and_oracle(n_a, Et, kw):
    V, T = cube_mesh(n_a)
    ops = {e: P.Operator(V, T, 1.0, Et, precision=P.PFMM_MIXED, nf_engine=e, **kw)
           for e in (P.PFMM_NF_AUTO, P.PFMM_NF_CUDA_CORES)}
    assert ops[P.PFMM_NF_AUTO].info()["nf_tensor_cores"] == 3
    assert ops[P.PFMM_NF_CUDA_CORES].info()["nf_tensor_cores"] == 0
    Pr = O.make_problem(V, T, 1.0, Et, **kw)
    w = random_density(Et, T.shape[0], 2, seed=21)
    g = random_density(Et, V.shape[0], 2, seed=22)
    for op_id, x in ((0, w), (1, g)):
        xt = torch.tensor(x, device=DEV)
        res = {}
        for e, o in ops.items():
            res[e] = (o.V(xt, parts=P.PFMM_PART_NEAR) if op_id == 0 else o.K(xt, parts=P.PFMM_PART_NEAR)).cpu().numpy()
            P.pfmm_check(o.h)
        # no atomics: the tensor-core product is bitwise reproducible
        o = ops[P.PFMM_NF_AUTO]
        again = (o.V(xt, parts=P.PFMM_PART_NEAR) if op_id == 0 else o.K(xt, parts=P.PFMM_PART_NEAR)).cpu().numpy()
        assert np.array_equal(again, res[P.PFMM_NF_AUTO])
        for r in range(2):
            ref = O.pfmm_apply(Pr, op_id, x[r], parts=1)
            assert _rel(res[P.PFMM_NF_AUTO][r], ref) <= 1e-5
            assert _rel(res[P.PFMM_NF_CUDA_CORES][r], ref) <= 1e-5
            assert _rel(res[P.PFMM_NF_AUTO][r], res[P.PFMM_NF_CUDA_CORES][r]) <= 1e-5
    for o in ops.values():
        o.close()


def test_tensor_core_split_scales_are_exact_powers_of_two():
    """The FP16 split scales each rhs by 2^E from its own max |x| and unscales exactly: an input
    multiplied by 2^k (any k within the FP32 range) gives the same FP16 parts, and the FP64 partial
    sums are added in a fixed order, so the nearfield of 2^k x is exactly 2^k times that of x; an
    all-zero rhs gives zeros, whatever the other right-hand sides hold."""
    V, T = cube_mesh(8)
    Et = 64
    op = P.Operator(V, T, 1.0, Et, m_t=4, m_x=6, c_st=1.0, precision=P.PFMM_MIXED)
    assert op.info()["nf_tensor_cores"] == 3
    w = random_density(Et, T.shape[0], 1, seed=31)[0]
    g = random_density(Et, V.shape[0], 1, seed=32)[0]
    for apply, x in ((op.V, w), (op.K, g)):
        # one call (the split-K chunking depends on the number of right-hand sides)
        k = [-80, 0, 80]
        xs = np.stack([np.ldexp(x, k[0]), x, np.ldexp(x, k[2]), np.zeros_like(x)])
        out = apply(torch.tensor(xs, device=DEV), parts=P.PFMM_PART_NEAR).cpu().numpy()
        P.pfmm_check(op.h)
        base = out[1]
        assert np.max(np.abs(base)) > 0
        for r in (0, 2):
            assert np.array_equal(np.ldexp(out[r], -k[r]), base)
        assert not np.any(out[3])
    op.close()


def test_dense_column_layout_with_holes():
    """Interaction areas that cover most but not all of the mesh (8^3-like leaf grid, n_tr = 6):
    the panels share one column space with zero (hole) columns for sources outside the area.
    FP64 against the oracle on sampled rows; mixed precision on the tensor cores against the
    CUDA-core engine on the same blocks."""
    V, T = cube_sphere_mesh(16)  # 3072 triangles
    Et = 64
    kw = dict(m_t=4, m_x=5, c_st=0.1, n_tr=6)
    op = P.Operator(V, T, 1.0, Et, **kw)
    info = op.info()
    assert info["nf_dense_columns"] == 1 and info["p"] == 5
    Pr = O.make_problem(V, T, 1.0, Et, **kw)
    w = random_density(Et, len(T), 1, seed=41)
    g = random_density(Et, len(V), 1, seed=42)
    rows = sample_triangles(len(T), 5, seed=43)
    fV = op.V(torch.tensor(w, device=DEV))[0].cpu().numpy()
    fK = op.K(torch.tensor(g, device=DEV))[0].cpu().numpy()
    assert _rel(fV, O.pfmm_apply(Pr, 0, w[0], targets=rows), rows) <= 1e-12
    assert _rel(fK, O.pfmm_apply(Pr, 1, g[0], targets=rows), rows) <= 1e-12
    op.close()
    opt = P.Operator(V, T, 1.0, Et, precision=P.PFMM_MIXED, **kw)
    opc = P.Operator(V, T, 1.0, Et, precision=P.PFMM_MIXED, nf_engine=P.PFMM_NF_CUDA_CORES, **kw)
    assert opt.info()["nf_tensor_cores"] == 3 and opc.info()["nf_tensor_cores"] == 0
    wt, gt = torch.tensor(w, device=DEV), torch.tensor(g, device=DEV)
    assert _rel(opt.V(wt).cpu().numpy(), opc.V(wt).cpu().numpy()) <= 1e-5
    assert _rel(opt.K(gt).cpu().numpy(), opc.K(gt).cpu().numpy()) <= 1e-5
    opt.close()
    opc.close()

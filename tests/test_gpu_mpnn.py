"""Learned preconditioner through the C ABI: forward and gradient against the CPU oracle
(oracle/mpnn.py, FP64, same bfloat16-rounded weights), the (residual, error) pairs recorded by
pfmm_solve against the operator, training, and FGMRES with the network as right preconditioner
(convergence judged by the exact operator, fallback to plain FGMRES)."""
import numpy as np
import pytest
import torch

import oracle as O_dense
from oracle import mpnn as O
from paper_2106_15911_gb300 import pfmm as P
from paper_2106_15911_gb300.inputs import cube_mesh, heat_source_datum, random_density, shell_sources

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("width,layers,n_a", [(64, 4, 2), (32, 2, 2), (16, 3, 2), (16, 0, 2), (64, 2, 4)])
def test_forward_matches_oracle(width, layers, n_a):
    V, T = cube_mesh(n_a, "cross")  # 96 / 384 triangles: tiles of 64 / 128 rows with ragged tails
    Et, nvec, c = 5, 2, 1.3
    net = P.Mpnn(V, T, 1.0, Et, width=width, layers=layers, seed=1)
    p = (np.random.default_rng(21).standard_normal(net.num_params()) * 0.3).astype(np.float32)
    net.set_params(p)
    net.output_scale = c
    v = random_density(Et, len(T), nvec, seed=22)
    v[1, 3] *= 1e-6  # a slice of a very different scale
    z = torch.empty((nvec, Et, len(T)), dtype=torch.float64, device=DEV)
    net.apply(torch.tensor(v, device=DEV), z)
    torch.cuda.synchronize()
    net.check()
    want = O.forward(O.bf16_round(p), width, layers, V, T, Et, c, v)
    got = z.cpu().numpy()
    # widths 32 and 64 run the layers on the tensor cores with the layer input split into BF16
    # hi + lo parts (about 16 significant bits); width 16 is FP32 on the CUDA cores
    tol = 1e-4
    for r in range(nvec):
        for t in range(Et):
            assert _rel(got[r, t], want[r, t]) <= tol, (r, t)
    net.close()


@pytest.mark.parametrize("width,tol", [(64, 1e-3), (16, 1e-3)])
def test_gradient_matches_oracle(width, tol):
    V, T = cube_mesh(2, "cross")
    Et, layers, c = 4, 4, 0.7
    net = P.Mpnn(V, T, 1.0, Et, width=width, layers=layers, seed=2)
    p = (np.random.default_rng(31).standard_normal(net.num_params()) * 0.2).astype(np.float32)
    net.set_params(p)
    net.output_scale = c
    R = random_density(Et, len(T), 2, seed=32)
    E = random_density(Et, len(T), 2, seed=33)
    slices = np.array([0, 5, 7, 2, 5], dtype=np.int32)  # repeated slice counts twice
    loss, g = net.loss_grad(torch.tensor(R, device=DEV), torch.tensor(E, device=DEV), slices)  # error form
    A = O.mean_matrix(O.edge_adjacency(T))
    feat = O.features(V, T)
    Rs = [R.reshape(-1, len(T))[s] for s in slices]
    Es = [E.reshape(-1, len(T))[s] for s in slices]
    want_l, want_g = O.loss_and_grad(O.bf16_round(p), width, layers, A, feat, Rs, Es, [s % Et for s in slices], Et, c)
    assert loss == pytest.approx(want_l, rel=tol / 2)
    assert np.max(np.abs(g - want_g)) <= tol * np.max(np.abs(want_g))
    net.close()


def _small_same_step_case():
    """96 triangles, 4 steps: one spatial box and no M2L level, so the stored nearfield block of
    offset 0 is the whole same-step block A_0, which the oracle assembles densely."""
    V, T = cube_mesh(2, "cross")
    Et = 4
    op = P.Operator(V, T, 1.0, Et, m_t=4, m_x=4, c_st=1.0)
    assert op.info()["p"] < 2
    A0 = O_dense.assemble_V(V, T, 1.0 / Et, nd=1)[0]
    return V, T, Et, op, A0


def test_same_step_gradient_matches_oracle():
    V, T, Et, op, A0 = _small_same_step_case()
    width, layers, c = 32, 3, 5.0
    net = P.Mpnn(V, T, 1.0, Et, width=width, layers=layers, seed=7)
    p = (np.random.default_rng(41).standard_normal(net.num_params()) * 0.2).astype(np.float32)
    net.set_params(p)
    net.output_scale = c
    R = random_density(Et, len(T), 2, seed=42)
    slices = np.array([1, 6, 3], dtype=np.int32)
    loss, g = net.loss_grad(torch.tensor(R, device=DEV), None, slices, handle=op.h)
    A = O.mean_matrix(O.edge_adjacency(T))
    Rs = [R.reshape(-1, len(T))[s] for s in slices]
    want_l, want_g = O.loss_and_grad(O.bf16_round(p), width, layers, A, O.features(V, T), Rs, None,
                                     [s % Et for s in slices], Et, c, A0)
    assert loss == pytest.approx(want_l, rel=1e-4)
    # the device gradient applies A_0 for A_0^T: equal up to the singular rules' asymmetry
    assert np.max(np.abs(A0 - A0.T)) <= 1e-4 * np.max(np.abs(A0))
    assert np.max(np.abs(g - want_g)) <= 2e-3 * np.max(np.abs(want_g))
    net.close()
    op.close()


@pytest.fixture(scope="module")
def recorded():
    """Pairs recorded by plain FGMRES on the 192-triangle cube, 16 steps, 6 data sets."""
    V, T = cube_mesh(4)
    Et, n = 16, 16 * 192
    op = P.Operator(V, T, 1.0, Et, m_t=4, m_x=6, c_st=1.0)
    cap = 60
    R = torch.zeros((cap, Et, len(T)), dtype=torch.float64, device=DEV)
    E = torch.zeros_like(R)
    used, sols = 0, []
    for k in range(6):
        g = torch.tensor(heat_source_datum(V, 1.0, Et, shell_sources(1, seed=400 + k))[None], device=DEV)
        x = torch.empty((1, Et, len(T)), dtype=torch.float64, device=DEV)
        o = P.pfmm_default_solve_opts()
        o.rec_r, o.rec_e = R[used].data_ptr(), E[used].data_ptr()
        o.rec_cap, o.rec_every = cap - used, 4
        info = P.pfmm_solve(op.h, P.PFMM_DIRECT, g, x, 1, o)
        assert info["rel_res"] <= 1e-8 and info["recorded"] >= 2
        sols.append((g, x, used, info["recorded"]))
        used += info["recorded"]
    yield V, T, Et, op, R, E, used, sols
    op.close()


def test_recorded_pairs_are_residual_error_pairs(recorded):
    V, T, Et, op, R, E, used, sols = recorded
    for g, x, first, cnt in sols:
        b = 0.5 * op.M(g) + op.K(g)
        bn = float(torch.linalg.norm(b))
        for k in range(first, first + cnt):
            xk = x[0] - E[k]
            rk = b[0] - op.V(xk)  # the residual of the stored iterate, recomputed
            assert float(torch.linalg.norm(rk - R[k])) <= 1e-10 * bn, k
            assert float(torch.linalg.norm(R[k])) > 100 * 1e-8 * bn  # only above the recording floor


@pytest.mark.parametrize("same_step", [False, True])
def test_training_lowers_the_loss_and_preconditions(recorded, same_step):
    V, T, Et, op, R, E, used, sols = recorded
    net = P.Mpnn(V, T, 1.0, Et, width=64, layers=4, seed=3)
    hist = net.train(R, E, used, steps=600, batch_slices=32, lr=3e-3, seed=4, handle=op.h if same_step else None)
    assert np.all(np.isfinite(hist))
    assert hist[-30:].mean() < 0.7 * hist[:10].mean()
    assert net.output_scale > 0
    # preconditioned FGMRES on a held-out datum: the exact operator judges the residual
    g = torch.tensor(heat_source_datum(V, 1.0, Et, shell_sources(1, seed=999))[None], device=DEV)
    x = torch.empty((1, Et, len(T)), dtype=torch.float64, device=DEV)
    o = P.pfmm_default_solve_opts()
    o.precond = net.ptr
    info = P.pfmm_solve(op.h, P.PFMM_DIRECT, g, x, 1, o)
    assert info["rel_res"] <= 1e-8 and info["precond_off"] == 0
    b = 0.5 * op.M(g) + op.K(g)
    assert float(torch.linalg.norm(b - op.V(x))) <= 1.01e-8 * float(torch.linalg.norm(b))
    plain = P.pfmm_solve(op.h, P.PFMM_DIRECT, g, torch.empty_like(x), 1)
    if same_step:
        # trained towards the same-step inverse A_0^{-1}, the (linear) network is a block-Jacobi-
        # like preconditioner: fewer FGMRES iterations than without it (exact block Jacobi halves
        # them on this mesh, a first-degree polynomial in the mean adjacency removes 28 %)
        assert info["iterations"] < 0.85 * plain["iterations"], (info["iterations"], plain["iterations"])
    net.close()


def test_non_finite_network_falls_back_to_plain_fgmres(recorded):
    V, T, Et, op, R, E, used, sols = recorded
    net = P.Mpnn(V, T, 1.0, Et, width=16, layers=2, seed=5)
    net.set_params(np.full(net.num_params(), 1e30, dtype=np.float32))  # overflows to Inf in FP32
    net.output_scale = 1.0
    g, x_ref = sols[0][0], sols[0][1]
    x = torch.empty_like(x_ref)
    o = P.pfmm_default_solve_opts()
    o.precond = net.ptr
    info = P.pfmm_solve(op.h, P.PFMM_DIRECT, g, x, 1, o)
    assert info["precond_off"] >= 1 and info["rel_res"] <= 1e-8
    assert _rel(x.cpu().numpy(), x_ref.cpu().numpy()) <= 1e-6
    net.close()


def test_invalid_preconditioner_arguments(recorded):
    V, T, Et, op, R, E, used, sols = recorded
    other = P.Mpnn(V, T, 1.0, Et * 2, width=16, layers=1, seed=6)  # built for another step count
    o = P.pfmm_default_solve_opts()
    o.precond = other.ptr
    x = torch.empty_like(sols[0][1])
    with pytest.raises(P.PfmmError, match="another mesh"):
        P.pfmm_solve(op.h, P.PFMM_DIRECT, sols[0][0], x, 1, o)
    net = P.Mpnn(V, T, 1.0, Et, width=16, layers=1, seed=6)
    with pytest.raises(P.PfmmError, match="output scale"):
        net.apply(R[:1], torch.empty_like(R[:1]))
    with pytest.raises(P.PfmmError):
        P.Mpnn(V, T, 1.0, Et, width=48, layers=1)
    other.close()
    net.close()


@pytest.mark.parametrize("width,layers", [(64, 4), (16, 2), (32, 0)])
def test_compiled_form_equals_the_network(width, layers):
    """The assembled per-step sparse operators reproduce the network (and the oracle)."""
    V, T = cube_mesh(3, "cross")  # 216 triangles
    Et, nvec, c = 6, 2, 0.9
    net = P.Mpnn(V, T, 1.0, Et, width=width, layers=layers, seed=8)
    p = (np.random.default_rng(51).standard_normal(net.num_params()) * 0.3).astype(np.float32)
    net.set_params(p)
    net.output_scale = c
    v = torch.tensor(random_density(Et, len(T), nvec, seed=52), device=DEV)
    z_net = torch.empty_like(v)
    net.apply(v, z_net)
    net.compile()
    z_c = torch.empty_like(v)
    net.apply(v, z_c)
    torch.cuda.synchronize()
    a, b = z_c.cpu().numpy(), z_net.cpu().numpy()
    # two FP32 evaluations of one linear map (the assembled coefficients are FP32 roundings)
    assert _rel(a, b) <= 5e-5
    want = O.forward(O.bf16_round(p), width, layers, V, T, Et, c, v.cpu().numpy())
    assert _rel(a, want) <= 1e-4
    # a parameter change drops the compiled form: apply follows the new weights again
    net.set_params(2.0 * p)
    net.output_scale = c
    z2 = torch.empty_like(v)
    net.apply(v, z2)
    want2 = O.forward(O.bf16_round(2.0 * p), width, layers, V, T, Et, c, v.cpu().numpy())
    assert _rel(z2.cpu().numpy(), want2) <= 1e-4
    net.close()

"""Batches of independent problems (ragged meshes, step counts and right-hand-side counts)
through one captured CUDA graph equal the per-problem applies; the engine autotuner keeps
parity with the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2106_15911_gb300 import pfmm as P
from paper_2106_15911_gb300.inputs import cube_mesh, cube_sphere_mesh, random_density

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _problems(precision, seed=3):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(6):
        n_a = (2, 4)[i % 2]
        V, T = (cube_mesh if i % 3 else cube_sphere_mesh)(n_a)
        Et = (16, 32, 64)[i % 3]
        prm = P.pfmm_default_params()
        prm.precision = precision
        prm.m_t = 3
        prm = P.pfmm_autotune_params(V, T, 1.0, Et, base=prm, tol=1e-5, m_lo=3, m_hi=6)
        out.append((V, T, 1.0, Et, 1.0, prm, int(rng.integers(1, 4))))
    return out


@pytest.mark.parametrize("precision", [P.PFMM_FP64, P.PFMM_MIXED])
def test_batched_graph_equals_individual_applies(precision):
    probs = _problems(precision)
    B = P.Batch([p[:6] for p in probs])
    ws = [torch.tensor(random_density(p[3], p[1].shape[0], p[6], seed=10 + i), device=DEV) for i, p in enumerate(probs)]
    fs = [torch.empty_like(w) for w in ws]
    for rep in range(2):  # capture, then replay
        for f in fs:
            f.fill_(float("nan"))
        B.apply_V(ws, fs)
        torch.cuda.synchronize()
        for i, p in enumerate(probs):
            ref = torch.empty_like(ws[i])
            P.pfmm_apply_V(B.handle(i), ws[i], ref, ws[i].shape[0])
            torch.cuda.synchronize()
            a, b = fs[i].cpu().numpy(), ref.cpu().numpy()
            assert np.all(np.isfinite(a))
            assert np.max(np.abs(a - b)) / np.max(np.abs(b)) <= 1e-12
    # new buffers: the graph is captured again
    ws2 = [w * 2.0 for w in ws]
    fs2 = [torch.empty_like(w) for w in ws2]
    B.apply_V(ws2, fs2)
    torch.cuda.synchronize()
    for i in range(len(probs)):
        assert torch.allclose(fs2[i], 2.0 * fs[i], rtol=1e-12, atol=0)
    B.close()


def test_engine_autotune_keeps_oracle_parity():
    probs = _problems(P.PFMM_MIXED, seed=5)[:3]
    B = P.Batch([p[:6] for p in probs], tune_engines=True)
    for i, (V, T, Tend, Et, alpha, prm, nr) in enumerate(probs):
        w = torch.tensor(random_density(Et, T.shape[0], 1, seed=40 + i), device=DEV)
        f = torch.empty_like(w)
        P.pfmm_apply_V(B.handle(i), w, f, 1)
        Pr = O.make_problem(V, T, Tend, Et, m_t=prm.m_t, m_x=prm.m_x, c_st=prm.c_st)
        ref = O.pfmm_apply(Pr, 0, w.cpu().numpy()[0])
        got = f.cpu().numpy()[0]
        assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= 1e-5
    B.close()


def test_autotuner_picks_an_m2l_form_that_keeps_the_product():
    """Degree 8 on 4^3 grids: the autotuner times the sliced fused M2L against the three global
    passes (CUDA events) and keeps one; the tuned product equals that of an untuned handle of the
    same problem within FP32 accuracy, and pfmm_get_info reports the engines in use."""
    V, T = cube_mesh(8)
    Et = 256
    prm = P.pfmm_default_params()
    prm.precision = P.PFMM_MIXED
    prm.m_t, prm.m_x, prm.c_st = 4, 8, 1.0
    B = P.Batch([(V, T, 1.0, Et, 1.0, prm)], tune_engines=True)
    op = P.Operator(V, T, 1.0, Et, m_t=4, m_x=8, c_st=1.0, precision=P.PFMM_MIXED)
    eng = P.pfmm_get_info(B.handle(0))["m2l_engine"]
    assert set(eng[6:]) <= {P.PFMM_M2L_FUSED_SLICED, P.PFMM_M2L_THREE_PASS}, eng
    w = torch.tensor(random_density(Et, T.shape[0], 2, seed=77), device=DEV)
    f = torch.empty_like(w)
    P.pfmm_apply_V(B.handle(0), w, f, 2)
    ref = op.V(w)
    torch.cuda.synchronize()
    assert float((f - ref).abs().max() / ref.abs().max()) <= 1e-5
    op.close()
    B.close()

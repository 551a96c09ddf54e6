"""Representation formula u = V~ w - W g (Section 2) on the GPU through the C ABI against the
CPU oracle (same quadrature rule, exact time integrals): FP64 within 1e-12 of the largest value,
for interior and exterior points at several times (including t <= 0 and t beyond the last step),
two right-hand sides, and the single-layer potential alone (g = NULL)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2106_15911_gb300 import pfmm as P
from paper_2106_15911_gb300.inputs import cube_mesh, cube_sphere_mesh, random_density

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("mesh,n_a,Et,qr", [(cube_mesh, 4, 16, 3), (cube_sphere_mesh, 4, 32, 4)])
def test_repr_matches_oracle(mesh, n_a, Et, qr):
    V, T = mesh(n_a)
    op = P.Operator(V, T, 1.0, Et, m_t=3, m_x=3, c_st=1.0, quad_regular=qr)
    rng = np.random.default_rng(17)
    c = V.mean(axis=0)
    pts = np.concatenate([c + 0.2 * rng.standard_normal((12, 3)), c + np.array([[1.5, 0.1, 0.0], [0.0, -1.4, 0.3]])])
    ts = np.concatenate([rng.uniform(0.05, 1.0, 12), [0.0, 1.3]])  # t = 0 gives 0; t > T uses every step
    pts = np.concatenate([pts, ts[:, None]], axis=1)
    w = random_density(Et, T.shape[0], 2, seed=18)
    g = random_density(Et, V.shape[0], 2, seed=19)
    Pr = O.make_problem(V, T, 1.0, Et, n_r=qr)
    pt = torch.tensor(pts, device=DEV)
    u = torch.empty((2, pts.shape[0]), dtype=torch.float64, device=DEV)
    P.pfmm_eval_repr(op.h, torch.tensor(w, device=DEV), torch.tensor(g, device=DEV), pt, u, 2)
    us = torch.empty_like(u)
    P.pfmm_eval_repr(op.h, torch.tensor(w, device=DEV), None, pt, us, 2)
    torch.cuda.synchronize()
    u, us = u.cpu().numpy(), us.cpu().numpy()
    for r in range(2):
        ref = O.repr_eval(Pr, w[r], g[r], pts)
        refs = O.repr_eval(Pr, w[r], None, pts)
        assert np.max(np.abs(ref)) > 0 and ref[12] == 0.0 and u[r, 12] == 0.0
        assert np.max(np.abs(u[r] - ref)) <= 1e-12 * np.max(np.abs(ref))
        assert np.max(np.abs(us[r] - refs)) <= 1e-12 * np.max(np.abs(refs))
    op.close()

"""Pins of the learned-preconditioner oracle (oracle/mpnn.py) to facts outside itself:
bfloat16 rounding against torch's conversion, the edge adjacency of closed meshes, outward
normals of the cube, closed-form single-row outputs written with scalar loops, invariances of the
definition (linearity in the slice), and the gradient against central finite differences."""
import math

import numpy as np
import pytest

from oracle import mpnn as O
from paper_2106_15911_gb300.inputs import cube_mesh, random_density

torch = pytest.importorskip("torch")

TET_V = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
TET_T = np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]], dtype=np.int32)


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.integers(-8, 8, 5000),
                        [1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -1.0 - 2.0 ** -8, 0.0, 65504.0]]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(O.bf16_round(x), want)
    # ties go to the even mantissa: 1 + 2^-8 is halfway between 1 and 1 + 2^-7
    assert O.bf16_round(np.float32(1.0 + 2.0 ** -8))[()] == 1.0
    assert O.bf16_round(np.float32(1.0 + 3 * 2.0 ** -8))[()] == 1.0 + 2.0 ** -6


def test_adjacency_tetrahedron_and_cube():
    adj = O.edge_adjacency(TET_T)
    assert adj == [[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]]
    for split in ("diag", "cross"):
        V, T = cube_mesh(2, split)
        adj = O.edge_adjacency(T)
        assert all(len(a) == 3 for a in adj)  # closed 2-manifold: 3 edge neighbours each
        assert all(i in adj[j] for i in range(len(adj)) for j in adj[i])  # symmetric
        assert sum(len(a) for a in adj) == 3 * len(T)  # every edge shared by exactly two triangles
        A = O.mean_matrix(adj)
        assert np.allclose(A @ np.ones(len(T)), 1.0)  # the mean of a constant field is that constant


def test_features_cube():
    V, T = cube_mesh(3)
    f = O.features(V, T)
    assert np.allclose(f[:, 0], 1.0)  # uniform grid, equal areas
    cen = V[T].mean(axis=1)
    out = cen - 0.5
    # the normal is the axis of the face the centroid lies on, pointing away from the centre
    k = np.argmax(np.abs(out), axis=1)
    want = np.zeros_like(out)
    want[np.arange(len(k)), k] = np.sign(out[np.arange(len(k)), k])
    assert np.allclose(f[:, 1:], want)


def _rand_params(width, layers, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(O.n_params(width, layers)) * scale


def test_zero_layers_closed_form_single_row():
    W = 8
    p = _rand_params(W, 0, 1)
    d = O.unpack(p, W, 0)
    feat = O.features(TET_V, TET_T)
    A = O.mean_matrix(O.edge_adjacency(TET_T))
    v = np.array([0.3, -1.2, 2.0, 0.5])
    Et, t, c = 7, 3, 2.5
    z = O.forward_slice(p, W, 0, A, feat, v, t, Et, c)
    for i in range(4):
        f = [feat[i, 0], feat[i, 1], feat[i, 2], feat[i, 3], (t + 0.5) / Et]
        y = 0.0
        for o in range(W):
            a = d["bg"][o]
            for k in range(5):
                a += f[k] * d["Wg"][k][o]
            y += d["wo"][o] * a / (1.0 + math.exp(-a))
        # the slice scale cancels: z_i = c v_i (w_o . e_i)
        assert z[i] == pytest.approx(c * v[i] * y, rel=1e-13, abs=1e-13)


def test_one_layer_closed_form_tetrahedron():
    W = 4
    p = _rand_params(W, 1, 2)
    d = O.unpack(p, W, 1)
    feat = O.features(TET_V, TET_T)
    A = O.mean_matrix(O.edge_adjacency(TET_T))
    v = np.array([1.0, -0.5, 0.25, 2.0])
    Et, t, c = 4, 0, 1.0
    z = O.forward_slice(p, W, 1, A, feat, v, t, Et, c)
    sil = lambda a: a / (1.0 + math.exp(-a))  # noqa: E731
    h0 = []
    for i in range(4):
        f = [*feat[i], (t + 0.5) / Et]
        h0.append([v[i] * sil(d["bg"][o] + sum(f[k] * d["Wg"][k][o] for k in range(5))) for o in range(W)])
    L = d["layers"][0]
    for i in range(4):
        nbrs = [j for j in range(4) if j != i]  # every face of a tetrahedron touches the other three
        m = [sum(h0[j][k] for j in nbrs) / 3 for k in range(W)]
        h1 = [h0[i][o] + sum(h0[i][k] * L["Ws"][k][o] + m[k] * L["Wn"][k][o] for k in range(W)) for o in range(W)]
        y = sum(d["wo"][o] * h1[o] for o in range(W))
        assert z[i] == pytest.approx(c * y, rel=1e-12, abs=1e-12)


def test_linear_in_the_slice():
    """The map v -> z is linear: the slice scale cancels and nothing nonlinear acts on v."""
    V, T = cube_mesh(2)
    W, Lay = 8, 2
    p = _rand_params(W, Lay, 3)
    v1 = random_density(4, len(T), 1, seed=9)
    v2 = random_density(4, len(T), 1, seed=10)
    z1 = O.forward(p, W, Lay, V, T, 4, 1.7, v1)
    z2 = O.forward(p, W, Lay, V, T, 4, 1.7, v2)
    z3 = O.forward(p, W, Lay, V, T, 4, 1.7, 2.5 * v1 - 0.75 * v2)
    assert np.allclose(z3, 2.5 * z1 - 0.75 * z2, rtol=1e-11, atol=1e-11 * np.abs(z3).max())


@pytest.mark.parametrize("layers,same_step", [(0, False), (1, False), (3, False), (2, True)])
def test_gradient_finite_differences(layers, same_step):
    V, T = cube_mesh(1, "cross")  # 24 triangles
    W = 8
    A = O.mean_matrix(O.edge_adjacency(T))
    feat = O.features(V, T)
    rng = np.random.default_rng(11 + layers)
    p = _rand_params(W, layers, 4 + layers, 0.5)
    Rs = [rng.standard_normal(len(T)) for _ in range(3)]
    Es = [rng.standard_normal(len(T)) for _ in range(3)]
    steps = [0, 2, 5]
    Et, c = 6, 0.8
    # same-step form: a non-symmetric A_0 stand-in, so that a transpose mistake shows
    A0 = rng.standard_normal((len(T), len(T))) / len(T) + np.eye(len(T)) if same_step else None
    val, g = O.loss_and_grad(p, W, layers, A, feat, Rs, Es, steps, Et, c, A0)
    assert val == pytest.approx(O.loss(p, W, layers, A, feat, Rs, Es, steps, Et, c, A0), rel=1e-13)
    idx = rng.choice(p.size, size=min(p.size, 60), replace=False)
    idx = np.union1d(idx, [0, p.size - 1, O.NG * W])  # W_g, w_o, b_g entries
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (O.loss(p + e, W, layers, A, feat, Rs, Es, steps, Et, c, A0) -
              O.loss(p - e, W, layers, A, feat, Rs, Es, steps, Et, c, A0)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-8), i


def test_same_step_loss_vanishes_for_the_exact_inverse():
    """The same-step loss term and its derivative vanish at the exact correction z = A_0^{-1} r."""
    rng = np.random.default_rng(3)
    A0 = rng.standard_normal((10, 10)) + 5 * np.eye(10)
    r = rng.standard_normal(10)
    val, dz = O._slice_loss(np.linalg.solve(A0, r), r, None, A0)
    assert val == pytest.approx(0.0, abs=1e-24) and np.allclose(dz, 0.0, atol=1e-12)

"""CPU FP64 oracle of the learned preconditioner network (forward, loss, gradient).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` alone.  It shares no code with the CUDA path.

The network is not part of the paper's method (the paper solves with unpreconditioned GMRES,
Section 5); it is the message-passing preconditioner acting on time slices of a Krylov vector.
Definition, for a slice v (E_x values of step t), s = RMS(v) + 1e-30, and the geometry / step
features f_i = (|gamma_i| / mean area, n_i, (t + 1/2) / E_t):

    e_i     = SiLU(f_i W_g + b_g)
    h^0_i   = (v_i / s) e_i
    h^{l+1} = h^l + h^l W_s^l + (A h^l) W_n^l,   (A h)_i = mean of h_j, j ~ i
    z_i     = c s (h^L_i . w_o)

j ~ i when triangles i and j share an edge.  Matrices are input-major (M[k][o] multiplies input
k into output o).  z is linear in v.  Two losses over S residual slices r_b:

* error form, with targets e_b:   (1/S) sum_b ||z(r_b) - e_b||^2 / (||e_b||^2 + 1e-30)
* same-step form, with the same-step block A_0 of V_h (dense here):
                                  (1/S) sum_b ||A_0 z(r_b) - r_b||^2 / (||r_b||^2 + 1e-30)

The gradient is the chain rule written out (``loss_and_grad``, with the exact transpose A_0^T);
it is pinned against central finite differences of ``loss``.

Weights enter the CUDA path in bfloat16; ``bf16_round`` is IEEE round-to-nearest-even of a
float32 to the 8-bit-mantissa format, so a test can hand both sides the same weight values.
"""
from __future__ import annotations

import numpy as np

NG = 5


def bf16_round(x) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


def edge_adjacency(triangles) -> list[list[int]]:
    """Neighbour lists: triangles sharing an edge (each neighbour once, sorted)."""
    owners: dict[tuple[int, int], list[int]] = {}
    for t, tri in enumerate(np.asarray(triangles)):
        for e in range(3):
            a, b = int(tri[e]), int(tri[(e + 1) % 3])
            owners.setdefault((min(a, b), max(a, b)), []).append(t)
    nb: list[set[int]] = [set() for _ in range(len(triangles))]
    for ts in owners.values():
        for a in ts:
            for b in ts:
                if a != b:
                    nb[a].add(b)
    return [sorted(s) for s in nb]


def mean_matrix(adj) -> np.ndarray:
    """Dense A with (A h)_i = mean over the neighbours of i (zero row when i has none)."""
    n = len(adj)
    A = np.zeros((n, n))
    for i, js in enumerate(adj):
        for j in js:
            A[i, j] = 1.0 / len(js)
    return A


def features(vertices, triangles) -> np.ndarray:
    """[E_x, 4]: area / mean area, outward unit normal (right-hand rule of the vertex order)."""
    V = np.asarray(vertices, dtype=np.float64)
    T = np.asarray(triangles)
    c = np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]])
    ln = np.linalg.norm(c, axis=1)
    area = 0.5 * ln
    out = np.empty((len(T), 4))
    out[:, 0] = area / area.mean()
    out[:, 1:] = c / ln[:, None]
    return out


def n_params(width: int, layers: int) -> int:
    return NG * width + width + layers * 2 * width * width + width


def unpack(p, width: int, layers: int) -> dict:
    """Split the flat parameter vector into named arrays (the layout of the CUDA path)."""
    p = np.asarray(p, dtype=np.float64)
    W = width
    o = 0

    def take(n, shape):
        nonlocal o
        a = p[o:o + n].reshape(shape)
        o += n
        return a

    d = {"Wg": take(NG * W, (NG, W)), "bg": take(W, (W,)), "layers": []}
    for _ in range(layers):
        d["layers"].append({"Ws": take(W * W, (W, W)), "Wn": take(W * W, (W, W))})
    d["wo"] = take(W, (W,))
    assert o == p.size
    return d


def silu(x):
    return x / (1.0 + np.exp(-x))


def dsilu(x):
    s = 1.0 / (1.0 + np.exp(-x))
    return s * (1.0 + x * (1.0 - s))


def slice_inputs(v, step: int, Et: int, feat) -> tuple[np.ndarray, np.ndarray, float]:
    """(v / s, the feature matrix F [E_x, 5], s) of one slice."""
    v = np.asarray(v, dtype=np.float64)
    s = float(np.sqrt(np.mean(v * v))) + 1e-30
    F = np.empty((v.size, NG))
    F[:, :4] = feat
    F[:, 4] = (step + 0.5) / Et
    return v / s, F, s


def forward_slice(p, width, layers, A, feat, v, step, Et, c, cache=None) -> np.ndarray:
    d = unpack(p, width, layers)
    x0, F, s = slice_inputs(v, step, Et, feat)
    P0 = F @ d["Wg"] + d["bg"]
    H = [x0[:, None] * silu(P0)]
    for lay in d["layers"]:
        H.append(H[-1] + H[-1] @ lay["Ws"] + (A @ H[-1]) @ lay["Wn"])
    y = H[-1] @ d["wo"]
    if cache is not None:
        cache.update(x0=x0, F=F, s=s, H=H, P0=P0, d=d)
    return c * s * y


def forward(p, width, layers, vertices, triangles, Et, c, V) -> np.ndarray:
    """z for every slice of V ([n_vec, E_t, E_x]); slices are independent."""
    A = mean_matrix(edge_adjacency(triangles))
    feat = features(vertices, triangles)
    V = np.asarray(V, dtype=np.float64)
    Z = np.empty_like(V)
    for r in range(V.shape[0]):
        for t in range(V.shape[1]):
            Z[r, t] = forward_slice(p, width, layers, A, feat, V[r, t], t, Et, c)
    return Z


def _slice_loss(z, r, e, A0):
    """Loss term of one slice and its derivative w.r.t. z (before the 1/S factor)."""
    r = np.asarray(r, dtype=np.float64)
    if A0 is None:
        e = np.asarray(e, dtype=np.float64)
        den = float(np.sum(e * e)) + 1e-30
        return float(np.sum((z - e) ** 2)) / den, 2.0 * (z - e) / den
    u = A0 @ z
    den = float(np.sum(r * r)) + 1e-30
    return float(np.sum((u - r) ** 2)) / den, A0.T @ (2.0 * (u - r) / den)


def loss(p, width, layers, A, feat, Rs, Es, steps, Et, c, A0=None) -> float:
    """Mean over the slices of the error-form loss (A0 None) or the same-step form."""
    tot = 0.0
    for b, (r, t) in enumerate(zip(Rs, steps)):
        z = forward_slice(p, width, layers, A, feat, r, t, Et, c)
        tot += _slice_loss(z, r, None if Es is None else Es[b], A0)[0]
    return tot / len(Rs)


def loss_and_grad(p, width, layers, A, feat, Rs, Es, steps, Et, c, A0=None) -> tuple[float, np.ndarray]:
    """Loss and its gradient w.r.t. the flat parameter vector (chain rule, layer by layer)."""
    S = len(Rs)
    W = width
    g = {"Wg": np.zeros((NG, W)), "bg": np.zeros(W), "wo": np.zeros(W),
         "layers": [{"Ws": np.zeros((W, W)), "Wn": np.zeros((W, W))} for _ in range(layers)]}
    tot = 0.0
    for b, (r, t) in enumerate(zip(Rs, steps)):
        cache: dict = {}
        z = forward_slice(p, width, layers, A, feat, r, t, Et, c, cache)
        val, dz = _slice_loss(z, r, None if Es is None else Es[b], A0)
        tot += val
        dy = dz / S * c * cache["s"]
        d, H = cache["d"], cache["H"]
        g["wo"] += H[-1].T @ dy
        G = np.outer(dy, d["wo"])
        for l in range(layers - 1, -1, -1):
            lay = d["layers"][l]
            g["layers"][l]["Ws"] += H[l].T @ G
            g["layers"][l]["Wn"] += (A @ H[l]).T @ G
            G = G + G @ lay["Ws"].T + A.T @ (G @ lay["Wn"].T)
        D = G * cache["x0"][:, None] * dsilu(cache["P0"])
        g["Wg"] += cache["F"].T @ D
        g["bg"] += D.sum(axis=0)
    parts = [g["Wg"].ravel(), g["bg"]]
    for gl in g["layers"]:
        parts += [gl["Ws"].ravel(), gl["Wn"].ravel()]
    parts.append(g["wo"])
    return tot / S, np.concatenate(parts)

"""Plain numpy solvers for the space-time system V_h w = (1/2 M_h + K_h) g (Section 2,
Eq. 02:linear:system).  TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* ``gmres``: restarted GMRES with modified Gram-Schmidt and Givens rotations (Saad & Schultz
  1986), x0 = 0, stopped on the relative residual ||b - A x|| / ||b|| (the paper solves the
  whole space-time system at once with unpreconditioned GMRES, Section 3 and Section 5).
* ``forward_substitution``: the unique exact solution of the block lower-triangular Toeplitz
  system (causality, Section 2): w_k = A_0^{-1} (b_k - sum_{d>=1} A_d w_{k-d}).  A_0 is solved
  by LU: it is symmetric positive definite in exact arithmetic, but the assembled block is
  symmetric only up to the singular quadrature's error, which a Cholesky factor (reading one
  triangle) would silently change.
"""
from __future__ import annotations

import numpy as np


def gmres(apply, b, tol=1e-8, restart=50, max_it=2000):
    """Solve apply(x) = b.  Returns (x, iterations, relative residual history)."""
    b = np.asarray(b, dtype=np.float64)
    shape = b.shape
    bv = b.ravel()
    nb = np.linalg.norm(bv)
    x = np.zeros_like(bv)
    hist = [1.0]
    if nb == 0.0:
        return x.reshape(shape), 0, hist
    it = 0
    while it < max_it:
        r = bv - apply(x.reshape(shape)).ravel()
        beta = np.linalg.norm(r)
        if beta / nb <= tol:
            break
        m = restart
        Q = np.zeros((m + 1, bv.size))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        Q[0] = r / beta
        j_end = 0
        for j in range(m):
            v = apply(Q[j].reshape(shape)).ravel()
            for i in range(j + 1):  # modified Gram-Schmidt
                H[i, j] = np.dot(Q[i], v)
                v = v - H[i, j] * Q[i]
            H[j + 1, j] = np.linalg.norm(v)
            if H[j + 1, j] > 0:
                Q[j + 1] = v / H[j + 1, j]
            for i in range(j):  # apply previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_end = j + 1
            hist.append(abs(g[j + 1]) / nb)
            if abs(g[j + 1]) / nb <= tol or it >= max_it:
                break
        y = np.linalg.solve(np.triu(H[:j_end, :j_end]), g[:j_end])
        x = x + Q[:j_end].T @ y
        if hist[-1] <= tol:
            r = bv - apply(x.reshape(shape)).ravel()
            if np.linalg.norm(r) / nb <= tol:
                break
    return x.reshape(shape), it, hist


def forward_substitution(blocks, b):
    """Exact solution of sum_{d=0}^{k} A_d w_{k-d} = b_k for k = 0..Et-1 (blocks [nd, n, n],
    blocks beyond nd are zero)."""
    import scipy.linalg

    lu = scipy.linalg.lu_factor(blocks[0])
    Et = b.shape[0]
    w = np.zeros_like(b, dtype=np.float64)
    for k in range(Et):
        rhs = b[k].copy()
        for d in range(1, min(k + 1, blocks.shape[0])):
            rhs -= blocks[d] @ w[k - d]
        w[k] = scipy.linalg.lu_solve(lu, rhs)
    return w

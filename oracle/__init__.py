"""CPU FP64 oracle for the space-time heat BEM operators and the pFMM matvec.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / ``--impl reference`` legs may import this package.  It shares no code with
the CUDA path in ``paper_2106_15911_gb300``; its arithmetic lives in ``pfmm_oracle.c`` (plain
C, FP64) and ``solve.py`` (plain numpy), each function citing the passage of arXiv 2106.15911
it follows.

Parity unpinned: the accuracy of the chosen nearfield quadrature rule against the paper's
semi-analytic scheme (not reproduced); it is pinned by self-convergence and by closed-form
Laplace potentials only.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pfmm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, IEEE semantics, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class Problem(ctypes.Structure):
    _fields_ = [
        ("nv", ctypes.c_int), ("nt", ctypes.c_int),
        ("V", ctypes.POINTER(ctypes.c_double)), ("T", ctypes.POINTER(ctypes.c_int)),
        ("Tend", ctypes.c_double), ("Et", ctypes.c_int), ("alpha", ctypes.c_double),
        ("m_t", ctypes.c_int), ("m_x", ctypes.c_int), ("c_st", ctypes.c_double),
        ("n_tr", ctypes.c_int), ("eps_tr", ctypes.c_double),
        ("leaf_steps", ctypes.c_int), ("leaf_tris", ctypes.c_int),
        ("n_r", ctypes.c_int), ("n_s", ctypes.c_int),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            d, i, pd, pi = ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
            for name in ("orc_G", "orc_G1", "orc_G2", "orc_G2t", "orc_DL2", "orc_DL2t"):
                getattr(L, name).restype = d
                getattr(L, name).argtypes = [d, d, d]
            for name in ("orc_time_V", "orc_time_K"):
                getattr(L, name).restype = d
                getattr(L, name).argtypes = [d, i, d, d]
            L.orc_gauss_legendre01.argtypes = [i, pd, pd]
            L.orc_pair_integral.argtypes = [pd, pi, pi, i, i, d, d, pd, i, i, pd]
            L.orc_assemble_V.argtypes = [i, pd, i, pi, d, d, i, i, i, i, pd, i]
            L.orc_assemble_K.argtypes = [i, pd, i, pi, d, d, i, i, i, i, pd, i]
            L.orc_assemble_V_rows.argtypes = [i, pd, i, pi, d, d, i, i, i, i, pi, i, pd, i]
            L.orc_assemble_M.argtypes = [i, pd, i, pi, d, pd]
            L.orc_tree_info.argtypes = [ctypes.POINTER(Problem), pi, pi, pi, pd, pi, pi, pd]
            L.orc_pfmm_apply.argtypes = [ctypes.POINTER(Problem), i, pd, pd, pi, i, i, i]
            L.orc_H1.restype = d
            L.orc_H1.argtypes = [d, d, d]
            L.orc_repr_eval.argtypes = [ctypes.POINTER(Problem), pd, pd, pd, i, pd, i]
            L.orc_E1.restype = d
            L.orc_E1.argtypes = [i, i, d, d, i]
            L.orc_space_moments.restype = i
            L.orc_space_moments.argtypes = [ctypes.POINTER(Problem), i, pd, d, i, pd]
            L.orc_time_moment.restype = d
            L.orc_time_moment.argtypes = [i, i, d, d, d, d]
            L.orc_qt.restype = d
            L.orc_qt.argtypes = [i, i, i, i]
            L.orc_qx.restype = d
            L.orc_qx.argtypes = [i, i, d, d, d, d, i]
            L.orc_lagrange.restype = d
            L.orc_lagrange.argtypes = [i, i, d, d, d]
            L.orc_cheb_node.restype = d
            L.orc_cheb_node.argtypes = [i, i]
            L.orc_interaction_list.argtypes = [i, pi]
            L.orc_nearfield_list.argtypes = [i, pi]
            L.orc_time_V_steps.restype = d
            L.orc_time_V_steps.argtypes = [d, d, d, d, d, d]
            L.orc_gen_tree_info.argtypes = [ctypes.POINTER(Problem), pd, i, pi, pi, pi, pi, pi, pi, pi, pi, pd, pi, i]
            L.orc_gen_interval.argtypes = [ctypes.POINTER(Problem), pd, i, i, i, pi, pi]
            L.orc_gen_coverage.argtypes = [ctypes.POINTER(Problem), pd, i, pi]
            L.orc_gen_pfmm_apply.argtypes = [ctypes.POINTER(Problem), pd, i, pd, pd, pi, i, i, i]
            L.orc_gen_dense_apply.argtypes = [ctypes.POINTER(Problem), pd, pd, pi, i, pd, i]
            L.orc_sizeof_problem.restype = i
            assert L.orc_sizeof_problem() == ctypes.sizeof(Problem)
            _lib = L
    return _lib


def _pd(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _pi(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


# ---- scalar kernels (Section 2) ------------------------------------------------------------
def G(r, s, alpha=1.0):
    return lib().orc_G(r, s, alpha)


def G1(r, s, alpha=1.0):
    return lib().orc_G1(r, s, alpha)


def G2(r, s, alpha=1.0):
    return lib().orc_G2(r, s, alpha)


def G2t(r, s, alpha=1.0):
    return lib().orc_G2t(r, s, alpha)


def DL2(r, s, alpha=1.0):
    return lib().orc_DL2(r, s, alpha)


def DL2t(r, s, alpha=1.0):
    return lib().orc_DL2t(r, s, alpha)


def time_V(r, d, h, alpha=1.0):
    return lib().orc_time_V(r, d, h, alpha)


def time_K(r, d, h, alpha=1.0):
    return lib().orc_time_K(r, d, h, alpha)


def gauss_legendre01(n):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().orc_gauss_legendre01(n, _pd(x), _pd(w))
    return x, w


KIND_V, KIND_K, KIND_LAPSL, KIND_LAPDL, KIND_POLY = 0, 1, 2, 3, 4


def pair_integral(V, tx, ty, kind, n, use_ss=True, d=0, h=1.0, alpha=1.0, poly=(0, 0, 0, 0)):
    """Integral over gamma_tx x gamma_ty of the chosen kernel (see pfmm_oracle.c, Sec. 3)."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    tx = np.ascontiguousarray(tx, dtype=np.int32)
    ty = np.ascontiguousarray(ty, dtype=np.int32)
    pc = np.ascontiguousarray(poly, dtype=np.float64)
    out = np.zeros(3)
    nc = lib().orc_pair_integral(_pd(V), _pi(tx), _pi(ty), kind, d, h, alpha, _pd(pc), n, 1 if use_ss else 0, _pd(out))
    return out[:nc] if nc > 1 else float(out[0])


# ---- dense Galerkin blocks (Section 2) -----------------------------------------------------
def assemble_V(V, T, h, alpha=1.0, d0=0, nd=1, n_r=3, n_s=6, nthreads=0):
    """Toeplitz blocks A_d[x][y] = V[(k,x),(k-d,y)], d = d0 .. d0+nd-1, shape [nd, nt, nt]."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.int32)
    out = np.zeros((nd, T.shape[0], T.shape[0]))
    rc = lib().orc_assemble_V(V.shape[0], _pd(V), T.shape[0], _pi(T), h, alpha, d0, nd, n_r, n_s, _pd(out), nthreads)
    assert rc == 0
    return out


def assemble_V_rows(V, T, h, rows, alpha=1.0, d0=0, nd=1, n_r=3, n_s=6, nthreads=0):
    """Rows of the Toeplitz blocks for the listed target triangles: A_d[rows[i]][y],
    d = d0 .. d0+nd-1, shape [nd, len(rows), nt] (nd <= 64 per call)."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.int32)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    out = np.zeros((nd, rows.shape[0], T.shape[0]))
    rc = lib().orc_assemble_V_rows(V.shape[0], _pd(V), T.shape[0], _pi(T), h, alpha, d0, nd, n_r, n_s, _pi(rows),
                                   rows.shape[0], _pd(out), nthreads)
    assert rc == 0
    return out


def toeplitz_rows_apply(blocks, x, leaf_steps=None):
    """f[k][i] = sum_{d} blocks[d][i] . x[k-d] for row blocks [nd, nrows, ncol] and x [Et, ncol]:
    the sampled rows of the block lower triangular Toeplitz product, shape [Et, nrows].  Without
    leaf_steps every d < min(k+1, nd) enters (blocks beyond nd are zero); with leaf_steps = ls only
    the pFMM nearfield offsets of step k on a uniform-depth tree do, d <= ls + (k mod ls) (the
    source steps of leaf intervals I_{i-1} and I_i, Eq. 03:ILtemp)."""
    Et = x.shape[0]
    f = np.zeros((Et, blocks.shape[1]))
    for k in range(Et):
        dmax = min(k + 1, blocks.shape[0])
        if leaf_steps:
            dmax = min(dmax, leaf_steps + k % leaf_steps + 1)
        for d in range(dmax):
            f[k] += blocks[d] @ x[k - d]
    return f


def assemble_K(V, T, h, alpha=1.0, d0=0, nd=1, n_r=3, n_s=6, nthreads=0):
    """Toeplitz blocks B_d[x][i] = K[(k,x),(k-d,i)] (node columns), shape [nd, nt, nv]."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.int32)
    out = np.zeros((nd, T.shape[0], V.shape[0]))
    rc = lib().orc_assemble_K(V.shape[0], _pd(V), T.shape[0], _pi(T), h, alpha, d0, nd, n_r, n_s, _pd(out), nthreads)
    assert rc == 0
    return out


def assemble_M(V, T, h):
    """Mass block M[(k,x),(k,i)] = h |gamma_x| / 3 for i a vertex of gamma_x, shape [nt, nv]."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.int32)
    out = np.zeros((T.shape[0], V.shape[0]))
    lib().orc_assemble_M(V.shape[0], _pd(V), T.shape[0], _pi(T), h, _pd(out))
    return out


def toeplitz_apply(blocks, x):
    """f[k] = sum_{d=0}^{k} A_d x[k-d] for blocks [nd,nt,ncol] and x [Et,ncol] (block lower
    triangular Toeplitz product of Section 2; blocks beyond nd are taken as zero)."""
    Et = x.shape[0]
    f = np.zeros((Et, blocks.shape[1]))
    for k in range(Et):
        for d in range(min(k + 1, blocks.shape[0])):
            f[k] += blocks[d] @ x[k - d]
    return f


# ---- tree and pFMM (Sections 3.2 - 3.4) ----------------------------------------------------
def make_problem(V, T, Tend, Et, alpha=1.0, m_t=4, m_x=4, c_st=1.0, n_tr=-1, eps_tr=1e-12, leaf_steps=2,
                 leaf_tris=16, n_r=3, n_s=6):
    V = np.ascontiguousarray(V, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.int32)
    P = Problem(V.shape[0], T.shape[0], _pd(V), _pi(T), Tend, Et, alpha, m_t, m_x, c_st, n_tr, eps_tr, leaf_steps,
                leaf_tris, n_r, n_s)
    P._keep = (V, T)
    return P


def tree_info(P):
    p = ctypes.c_int()
    lx = np.zeros(32, np.int32)
    nbox = np.zeros(32, np.int32)
    pad = np.zeros(32)
    ntr = np.zeros(32, np.int32)
    ntn = ctypes.c_int()
    root = np.zeros(4)
    rc = lib().orc_tree_info(ctypes.byref(P), ctypes.byref(p), _pi(lx), _pi(nbox), _pd(pad), _pi(ntr),
                             ctypes.byref(ntn), _pd(root))
    if rc:
        raise ValueError("tree build failed")
    n = p.value + 1
    return dict(p=p.value, lx=lx[:n].tolist(), nbox=nbox[:n].tolist(), pad=pad[:n].tolist(),
                ntr_far=ntr[:n].tolist(), ntr_near=ntn.value, corner=root[:3].tolist(), H=float(root[3]))


def pfmm_apply(P, op, x, targets=None, parts=3, nthreads=0):
    """Oracle pFMM (Alg. 2): op 0 -> V_h w (x [Et,nt]), op 1 -> K_h g (x [Et,nv]).
    Returns f [Et, nt]; rows of triangles outside ``targets`` are zero."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    f = np.zeros((P.Et, P.nt))
    if targets is None:
        tg, nt = None, -1
    else:
        tg = np.ascontiguousarray(targets, dtype=np.int32)
        nt = tg.shape[0]
    rc = lib().orc_pfmm_apply(ctypes.byref(P), op, _pd(x), _pd(f), _pi(tg) if tg is not None else None, nt, parts,
                              nthreads)
    if rc:
        raise ValueError("oracle pfmm failed")
    return f


def H1(r, s, alpha=1.0):
    """int_0^s G(r, q) / (2 q) dq (the time integral of the double-layer kernel's factor)."""
    return lib().orc_H1(r, s, alpha)


def repr_eval(P, w, g, points, nthreads=0):
    """Representation formula u = V~ w - W g (Section 2) at points [np][4] = (x, y, z, t) for the
    discrete data w [Et][nt] (p0 in space and time) and g [Et][nv] (p1 in space, p0 in time; None:
    single-layer potential only)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 4)
    gg = None if g is None else np.ascontiguousarray(g, dtype=np.float64)
    u = np.zeros(pts.shape[0])
    rc = lib().orc_repr_eval(ctypes.byref(P), _pd(w), _pd(gg) if gg is not None else None, _pd(pts), pts.shape[0],
                             _pd(u), nthreads)
    if rc:
        raise ValueError("oracle representation formula failed")
    return u


def interaction_list(k):
    """Temporal interaction list of interval k (Eq. 03:ILtemp), same-level indices."""
    js = np.zeros(2, np.int32)
    n = lib().orc_interaction_list(k, _pi(js))
    return js[:n].tolist()


def nearfield_list(k):
    """Temporal nearfield of interval k on a uniform-depth tree (Eq. 03:ILtemp)."""
    js = np.zeros(2, np.int32)
    n = lib().orc_nearfield_list(k, _pi(js))
    return js[:n].tolist()


def E1(k, l, r, dab, mx):
    return lib().orc_E1(k, l, r, dab, mx)


def space_moments(P, x, cen, hp, op=0):
    """Spatial moments of triangle x about the padded box (cen, hp) used by S2M / L2T (Eq. s2m,
    l2t): op 0 -> [n_kappa] values int_x T_{Y,kappa}; op 1 -> [n_kappa, 3] values
    int_x alpha n.grad T_{Y,kappa} phi_v.  Multi-indices with |kappa| <= m_x, kappa_1 slowest
    (``multi_indices``)."""
    nk = len(multi_indices(P.m_x))
    out = np.zeros(nk * (3 if op else 1))
    c = np.ascontiguousarray(cen, dtype=np.float64)
    n = lib().orc_space_moments(ctypes.byref(P), int(x), _pd(c), float(hp), int(op), _pd(out))
    assert n == nk
    return out.reshape(nk, 3) if op else out


def multi_indices(m):
    """The oracle's multi-index order: kappa with |kappa| <= m, kappa_1 slowest."""
    return [(a, b, c) for a in range(m + 1) for b in range(m + 1 - a) for c in range(m + 1 - a - b)]


def time_moment(a, m, jlo, jhi, lo, h):
    """int over (lo, lo + h] of the Lagrange polynomial L_{J,a} of the interval J = (jlo, jhi]."""
    return lib().orc_time_moment(a, m, jlo, jhi, lo, h)


def qt(c, ac, ap, m):
    return lib().orc_qt(c, ac, ap, m)


def qx(kap, nu, cc, hc, cp, hp, m):
    return lib().orc_qx(kap, nu, cc, hc, cp, hp, m)


def lagrange(b, m, lo, hi, t):
    return lib().orc_lagrange(b, m, lo, hi, t)


def cheb_node(k, m):
    return lib().orc_cheb_node(k, m)


# ---- general time steps (Section 3.2 with Alg. 1 in full, Section 3.3, Alg. 2) ---------------
def make_general_problem(V, T, ts, alpha=1.0, m_t=4, m_x=4, c_st=1.0, n_tr=-1, eps_tr=1e-12, n_r=3, n_s=6):
    """Problem for the time steps ts[0] = 0 < ts[1] < ... < ts[Et] = T (single layer)."""
    ts = np.ascontiguousarray(ts, dtype=np.float64)
    P = make_problem(V, T, float(ts[-1]), ts.shape[0] - 1, alpha=alpha, m_t=m_t, m_x=m_x, c_st=c_st, n_tr=n_tr,
                     eps_tr=eps_tr, n_r=n_r, n_s=n_s)
    P._ts = ts
    return P


def time_V_steps(r, tk0, tk1, tj0, tj1, alpha=1.0):
    """int over the target step (tk0, tk1] and the source step (tj0, tj1] of the heat kernel."""
    return lib().orc_time_V_steps(r, tk0, tk1, tj0, tj1, alpha)


def gen_tree_info(P, n_max, boxes=False):
    """The general tree: per level lx, boxes, leaves, intervals present, radii, refinement kind,
    padding; with boxes=True also [nbox_total][6] rows (level, cell x y z, k, leaf)."""
    nlev = ctypes.c_int()
    a = {k: np.zeros(32, np.int32) for k in ("lx", "nbox", "nleaf", "nint", "ntr_far", "ntr_near", "st")}
    pad = np.zeros(32)
    cap = 1 << 20 if boxes else 0
    bx = np.zeros((max(cap, 1), 6), np.int32)
    rc = lib().orc_gen_tree_info(ctypes.byref(P), _pd(P._ts), n_max, ctypes.byref(nlev), _pi(a["lx"]),
                                 _pi(a["nbox"]), _pi(a["nleaf"]), _pi(a["nint"]), _pi(a["ntr_far"]),
                                 _pi(a["ntr_near"]), _pi(a["st"]), _pd(pad), _pi(bx) if boxes else None, cap)
    if rc:
        raise ValueError("general tree build failed")
    n = nlev.value
    out = {k: v[:n].tolist() for k, v in a.items()}
    out["nlev"] = n
    out["pad"] = pad[:n].tolist()
    if boxes:
        out["boxes"] = bx[:sum(out["nbox"])]
    return out


def gen_interval(P, n_max, l, k):
    """Steps [ia, ib) of interval k of level l of the general tree ((-1, -1) when absent)."""
    ia, ib = ctypes.c_int(), ctypes.c_int()
    if lib().orc_gen_interval(ctypes.byref(P), _pd(P._ts), n_max, l, k, ctypes.byref(ia), ctypes.byref(ib)):
        raise ValueError("general tree build failed")
    return ia.value, ib.value


def gen_coverage(P, n_max):
    """cover[e, e'] (e = k nt + x target, e' = j nt + y source): how often the nearfield blocks and
    the admissible blocks of the general tree cover the pair (tiny problems only)."""
    ne = P.Et * P.nt
    cov = np.zeros((ne, ne), np.int32)
    if lib().orc_gen_coverage(ctypes.byref(P), _pd(P._ts), n_max, _pi(cov)):
        raise ValueError("general tree build failed")
    return cov


def gen_pfmm_apply(P, n_max, w, targets=None, parts=3, nthreads=0):
    """Oracle pFMM (Alg. 2) on the general tree: f = V_h w, w and f [Et, nt]."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    f = np.zeros((P.Et, P.nt))
    if targets is None:
        tg, n = None, -1
    else:
        tg = np.ascontiguousarray(targets, dtype=np.int32)
        n = tg.shape[0]
    rc = lib().orc_gen_pfmm_apply(ctypes.byref(P), _pd(P._ts), n_max, _pd(w), _pd(f),
                                  _pi(tg) if tg is not None else None, n, parts, nthreads)
    if rc:
        raise ValueError("oracle general pfmm failed")
    return f


def gen_dense_apply(P, w, targets, nthreads=0):
    """Dense Galerkin product V_h w on the rows of the listed triangles (all steps), general steps."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    tg = np.ascontiguousarray(targets, dtype=np.int32)
    f = np.zeros((P.Et, P.nt))
    lib().orc_gen_dense_apply(ctypes.byref(P), _pd(P._ts), _pd(w), _pi(tg), tg.shape[0], _pd(f), nthreads)
    return f

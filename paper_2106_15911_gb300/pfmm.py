"""Thin Python binding of the C ABI in include/pfmm.h (argument marshalling only).

Every function here forwards to the CUDA library ``libpfmm.so`` built in-tree by
``paper_2106_15911_gb300.build``; there is no CPU fallback: if the library is missing or a
call fails, an exception is raised.  Device vectors are passed as ``torch.Tensor`` (FP64,
CUDA, contiguous) or as raw integer device pointers; streams as ``torch.cuda.Stream`` or raw
``cudaStream_t`` integers (None = torch's current stream).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

PFMM_OK = 0
PFMM_ERR = {-1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "NONFINITE", -5: "TIMEOUT", -6: "NOT_CONVERGED",
            -7: "UNSUPPORTED"}
PFMM_FP64, PFMM_MIXED = 0, 1
PFMM_NEARFIELD_STORED, PFMM_NEARFIELD_ONTHEFLY = 0, 1
PFMM_PART_NEAR, PFMM_PART_FAR, PFMM_PART_ALL = 1, 2, 3
PFMM_NF_AUTO, PFMM_NF_CUDA_CORES = 0, 1
PFMM_M2L_THREE_PASS, PFMM_M2L_FUSED, PFMM_M2L_SLAB, PFMM_M2L_FUSED_SLICED = 1, 2, 3, 4


class pfmm_mesh(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int32), ("n_triangles", ctypes.c_int32),
                ("vertices", ctypes.POINTER(ctypes.c_double)), ("triangles", ctypes.POINTER(ctypes.c_int32)),
                ("T", ctypes.c_double), ("n_steps", ctypes.c_int32), ("alpha", ctypes.c_double)]


class pfmm_params(ctypes.Structure):
    _fields_ = [("m_t", ctypes.c_int32), ("m_x", ctypes.c_int32), ("c_st", ctypes.c_double),
                ("n_tr", ctypes.c_int32), ("eps_tr", ctypes.c_double), ("leaf_steps", ctypes.c_int32),
                ("leaf_tris", ctypes.c_int32), ("precision", ctypes.c_int32), ("nearfield", ctypes.c_int32),
                ("quad_regular", ctypes.c_int32), ("quad_singular", ctypes.c_int32), ("nf_engine", ctypes.c_int32),
                ("fp64_native", ctypes.c_int32), ("nf_form", ctypes.c_int32)]


class pfmm_gen_info(ctypes.Structure):
    _fields_ = [("nlev", ctypes.c_int32), ("lx", ctypes.c_int32 * 32), ("nbox", ctypes.c_int32 * 32),
                ("nleaf", ctypes.c_int32 * 32), ("nint", ctypes.c_int32 * 32), ("ntr_far", ctypes.c_int32 * 32),
                ("ntr_near", ctypes.c_int32 * 32), ("st", ctypes.c_int32 * 32), ("pad", ctypes.c_double * 32),
                ("n_m2l_pairs", ctypes.c_int64), ("n_near_blocks", ctypes.c_int64),
                ("nearfield_entries", ctypes.c_int64), ("device_bytes", ctypes.c_int64)]


class pfmm_info(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int32), ("lx", ctypes.c_int32 * 32), ("nbox", ctypes.c_int32 * 32),
                ("pad", ctypes.c_double * 32), ("n_m2l_pairs", ctypes.c_int32), ("nearfield_bytes", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("nf_tensor_cores", ctypes.c_int32),
                ("nearfield_v_elements", ctypes.c_int64), ("nf_dense_columns", ctypes.c_int32),
                ("m2l_engine", ctypes.c_int32 * 32), ("nf_form", ctypes.c_int32),
                ("nf_form_ms", ctypes.c_double * 2), ("m2l_flops", ctypes.c_double)]


class pfmm_solve_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int32), ("max_it", ctypes.c_int32),
                ("refine", ctypes.c_void_p), ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int32),
                ("precond", ctypes.c_void_p), ("rec_r", ctypes.c_void_p), ("rec_e", ctypes.c_void_p),
                ("rec_cap", ctypes.c_int32), ("rec_every", ctypes.c_int32), ("rec_basis", ctypes.c_int32)]


class pfmm_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("outer", ctypes.c_int32), ("rel_res", ctypes.c_double),
                ("seconds", ctypes.c_double), ("recorded", ctypes.c_int32), ("precond_off", ctypes.c_int32)]


PFMM_DIRECT, PFMM_INDIRECT = 0, 1

_lib = None
_lock = threading.Lock()

# (name, restype, argtypes) of every entry point declared in include/pfmm.h
_VP, _I, _DP = ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p
SIGNATURES = {
    "pfmm_default_params": (ctypes.c_int, [ctypes.POINTER(pfmm_params)]),
    "pfmm_build_trees": (ctypes.c_int, [ctypes.POINTER(pfmm_mesh), ctypes.POINTER(pfmm_params), _VP,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "pfmm_apply_V": (ctypes.c_int, [_VP, _DP, _DP, _I, _VP]),
    "pfmm_apply_K": (ctypes.c_int, [_VP, _DP, _DP, _I, _VP]),
    "pfmm_apply_M": (ctypes.c_int, [_VP, _DP, _DP, _I, _VP]),
    "pfmm_apply_parts": (ctypes.c_int, [_VP, _I, _DP, _DP, _I, _I, _VP]),
    "pfmm_apply_V_noalloc": (ctypes.c_int, [_VP, _DP, _DP, _I, _VP]),
    "pfmm_set_profiling": (ctypes.c_int, [_VP, _I]),
    "pfmm_phase_times": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)]),
    "pfmm_nf_kernel_time": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)]),
    "pfmm_get_info": (ctypes.c_int, [_VP, ctypes.POINTER(pfmm_info)]),
    "pfmm_gen_create": (ctypes.c_int, [ctypes.POINTER(pfmm_mesh), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(pfmm_params), _I, _VP, ctypes.POINTER(ctypes.c_void_p)]),
    "pfmm_gen_apply_V": (ctypes.c_int, [_VP, _DP, _DP, _I, _I, _VP]),
    "pfmm_gen_get_info": (ctypes.c_int, [_VP, ctypes.POINTER(pfmm_gen_info)]),
    "pfmm_gen_boxes": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int32), ctypes.c_int64,
                                      ctypes.POINTER(ctypes.c_int64)]),
    "pfmm_gen_destroy": (None, [_VP]),
    "pfmm_check": (ctypes.c_int, [_VP]),
    "pfmm_probe_fma_rate": (ctypes.c_int, [_I, ctypes.POINTER(ctypes.c_double), _VP]),
    "pfmm_eval_repr": (ctypes.c_int, [_VP, _DP, _DP, _DP, _I, _DP, _I, _VP]),
    "pfmm_shard_owners": (ctypes.c_int, [_I, _I, ctypes.POINTER(ctypes.c_int32)]),
    "pfmm_shard_messages": (ctypes.c_int, [_I, _I, ctypes.POINTER(ctypes.c_int32), ctypes.c_int64,
                                           ctypes.POINTER(ctypes.c_int64)]),
    "pfmm_count_apply_kernels": (ctypes.c_int, [_VP, _I, _DP, _DP, _I, _I, ctypes.POINTER(ctypes.c_int64)]),
    "pfmm_default_solve_opts": (ctypes.c_int, [ctypes.POINTER(pfmm_solve_opts)]),
    "pfmm_solve": (ctypes.c_int, [_VP, _I, _DP, _DP, _I, ctypes.POINTER(pfmm_solve_opts),
                                  ctypes.POINTER(pfmm_solve_info), _VP]),
    "pfmm_autotune_params": (ctypes.c_int, [ctypes.POINTER(pfmm_mesh), ctypes.POINTER(pfmm_params), ctypes.c_double,
                                            _I, _I, ctypes.POINTER(pfmm_params)]),
    "pfmm_build_trees_batched": (ctypes.c_int, [_I, ctypes.POINTER(pfmm_mesh), ctypes.POINTER(pfmm_params), _I, _VP,
                                                ctypes.POINTER(ctypes.c_void_p)]),
    "pfmm_apply_V_batched": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                            ctypes.POINTER(ctypes.c_int32), _VP]),
    "pfmm_batch_handle": (ctypes.c_int, [_VP, _I, ctypes.POINTER(ctypes.c_void_p)]),
    "pfmm_batch_size": (ctypes.c_int32, [_VP]),
    "pfmm_batch_set_streams": (ctypes.c_int, [_VP, _I]),
    "pfmm_batch_destroy": (None, [_VP]),
    "pfmm_mpnn_create": (ctypes.c_int, [ctypes.POINTER(pfmm_mesh), _I, _I, ctypes.c_uint64,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "pfmm_mpnn_num_params": (ctypes.c_int64, [_VP]),
    "pfmm_mpnn_get_params": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float), ctypes.c_int64]),
    "pfmm_mpnn_set_params": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float), ctypes.c_int64]),
    "pfmm_mpnn_set_output_scale": (ctypes.c_int, [_VP, ctypes.c_float]),
    "pfmm_mpnn_get_output_scale": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float)]),
    "pfmm_mpnn_apply": (ctypes.c_int, [_VP, _DP, _DP, _I, _VP]),
    "pfmm_mpnn_loss_grad": (ctypes.c_int, [_VP, _VP, _DP, _DP, ctypes.POINTER(ctypes.c_int32), _I,
                                           ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), _VP]),
    "pfmm_mpnn_train": (ctypes.c_int, [_VP, _VP, _DP, _DP, ctypes.c_int64, _I, _I, ctypes.c_float, ctypes.c_uint64,
                                       ctypes.POINTER(ctypes.c_float), _VP]),
    "pfmm_mpnn_check": (ctypes.c_int, [_VP]),
    "pfmm_mpnn_compile": (ctypes.c_int, [_VP, _VP]),
    "pfmm_mpnn_destroy": (None, [_VP]),
    "pfmm_destroy": (None, [_VP]),
    "pfmm_last_error": (ctypes.c_char_p, []),
}


def _preload_cudart():
    """Make libcudart resolvable for the dlopen of libpfmm.so (CUDA toolkit or torch's copy)."""
    for d in ("/usr/local/cuda/lib64", "/usr/local/cuda/targets/sbsa-linux/lib", "/usr/local/cuda/targets/x86_64-linux/lib"):
        for n in ("libcudart.so.13", "libcudart.so"):
            p = os.path.join(d, n)
            if os.path.exists(p):
                try:
                    ctypes.CDLL(p, mode=ctypes.RTLD_GLOBAL)
                    return
                except OSError:
                    pass


def lib(build_if_missing: bool = True):
    """Load libpfmm.so (building it first if needed).  Raises if it cannot be loaded."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                if not build_if_missing:
                    raise RuntimeError(f"CUDA library {path} is missing; run __graft_entry__.build()")
                path = _build.build()
            _preload_cudart()
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


class PfmmError(RuntimeError):
    pass


def _check(rc):
    if rc != PFMM_OK:
        msg = lib().pfmm_last_error().decode(errors="replace")
        raise PfmmError(f"pfmm error {rc} ({PFMM_ERR.get(rc, '?')}): {msg}")


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    import torch

    if isinstance(x, torch.Tensor):
        if not x.is_cuda or x.dtype != torch.float64 or not x.is_contiguous():
            raise ValueError("expected a contiguous float64 CUDA tensor")
        return x.data_ptr()
    raise TypeError(f"cannot pass {type(x)} as a device pointer")


def _stream(s):
    if isinstance(s, int):
        return s
    import torch

    if s is None:
        s = torch.cuda.current_stream()
    return s.cuda_stream


def pfmm_default_params() -> pfmm_params:
    p = pfmm_params()
    _check(lib().pfmm_default_params(ctypes.byref(p)))
    return p


def pfmm_build_trees(vertices, triangles, T, n_steps, alpha=1.0, params: pfmm_params | None = None, stream=None):
    """Build a handle (Alg. 1 tree, lists, tables, stored nearfield).  Returns an opaque handle."""
    V = np.ascontiguousarray(vertices, dtype=np.float64)
    Tr = np.ascontiguousarray(triangles, dtype=np.int32)
    m = pfmm_mesh(V.shape[0], Tr.shape[0], V.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                  Tr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), float(T), int(n_steps), float(alpha))
    if params is None:
        params = pfmm_default_params()
    h = ctypes.c_void_p()
    _check(lib().pfmm_build_trees(ctypes.byref(m), ctypes.byref(params), _stream(stream), ctypes.byref(h)))
    return h


def pfmm_apply_V(h, w, f, nrhs: int, stream=None):
    _check(lib().pfmm_apply_V(h, _ptr(w), _ptr(f), int(nrhs), _stream(stream)))


def pfmm_apply_K(h, g, f, nrhs: int, stream=None):
    _check(lib().pfmm_apply_K(h, _ptr(g), _ptr(f), int(nrhs), _stream(stream)))


def pfmm_apply_M(h, g, f, nrhs: int, stream=None):
    _check(lib().pfmm_apply_M(h, _ptr(g), _ptr(f), int(nrhs), _stream(stream)))


def pfmm_apply_V_noalloc(h, w, f, nrhs: int, stream=None):
    """f = V_h w with all workspaces in the library's static 64 MiB device array (no allocation)."""
    _check(lib().pfmm_apply_V_noalloc(h, _ptr(w), _ptr(f), int(nrhs), _stream(stream)))


def pfmm_apply_parts(h, op: int, x, f, nrhs: int, parts: int, stream=None):
    _check(lib().pfmm_apply_parts(h, int(op), _ptr(x), _ptr(f), int(nrhs), int(parts), _stream(stream)))


def pfmm_eval_repr(h, w, g, points, u, nrhs: int, stream=None):
    """u[rhs][p] = (V~ w - W g)(points[p]) (Section 2); g may be None (single layer only)."""
    _check(lib().pfmm_eval_repr(h, _ptr(w), _ptr(g), _ptr(points), int(points.shape[0]), _ptr(u), int(nrhs),
                                _stream(stream)))


PFMM_MSG_MOMENTS, PFMM_MSG_LOCALS, PFMM_MSG_INPUT = 0, 1, 2


def pfmm_shard_owners(levels: int, nranks: int):
    """Owner rank of every temporal cluster: a list per level l = 0 .. levels of 2^l ranks."""
    import numpy as np

    o = np.zeros((1 << (levels + 1)) - 1, np.int32)
    _check(lib().pfmm_shard_owners(int(levels), int(nranks), o.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    return [o[(1 << l) - 1:(1 << (l + 1)) - 1].tolist() for l in range(levels + 1)]


def pfmm_shard_messages(levels: int, nranks: int):
    """Messages of a distributed product: int array [n][5] of (kind, level, interval, src, dst)."""
    import numpy as np

    n = ctypes.c_int64()
    _check(lib().pfmm_shard_messages(int(levels), int(nranks), None, 0, ctypes.byref(n)))
    m = np.zeros((max(n.value, 1), 5), np.int32)
    _check(lib().pfmm_shard_messages(int(levels), int(nranks), m.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                     n.value, ctypes.byref(n)))
    return m[:n.value]


def pfmm_count_apply_kernels(h, op: int, x, f, nrhs: int, parts: int = PFMM_PART_ALL) -> int:
    """Kernels one pfmm_apply_parts call launches (counted in a captured graph, nothing runs)."""
    n = ctypes.c_int64()
    _check(lib().pfmm_count_apply_kernels(h, int(op), _ptr(x), _ptr(f), int(nrhs), int(parts), ctypes.byref(n)))
    return n.value


def pfmm_set_profiling(h, on: bool):
    _check(lib().pfmm_set_profiling(h, 1 if on else 0))


PHASES = ("permute_in", "nearfield", "s2m", "m2m", "m2l", "l2l", "l2t", "permute_out")


def pfmm_phase_times(h):
    ms = (ctypes.c_double * 8)()
    n = ctypes.c_int32()
    _check(lib().pfmm_phase_times(h, ms, ctypes.byref(n)))
    return dict(zip(PHASES, list(ms))), n.value


def pfmm_nf_kernel_time(h):
    """(milliseconds, launches) of the nearfield product kernel alone since the last call."""
    ms = ctypes.c_double()
    n = ctypes.c_int32()
    _check(lib().pfmm_nf_kernel_time(h, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def pfmm_get_info(h) -> dict:
    i = pfmm_info()
    _check(lib().pfmm_get_info(h, ctypes.byref(i)))
    n = i.p + 1
    return dict(p=i.p, lx=list(i.lx[:n]), nbox=list(i.nbox[:n]), pad=list(i.pad[:n]), n_m2l_pairs=i.n_m2l_pairs,
                nearfield_bytes=i.nearfield_bytes, device_bytes=i.device_bytes, nf_tensor_cores=i.nf_tensor_cores,
                nearfield_v_elements=i.nearfield_v_elements, nf_dense_columns=i.nf_dense_columns,
                m2l_engine=list(i.m2l_engine[:n]), nf_form=i.nf_form, nf_form_ms=list(i.nf_form_ms),
                m2l_flops=i.m2l_flops)


def pfmm_check(h):
    """Synchronise and raise if a bounded device wait of this handle gave up (TIMEOUT)."""
    _check(lib().pfmm_check(h))


def pfmm_probe_fma_rate(fp64: bool, stream=None) -> float:
    v = ctypes.c_double()
    _check(lib().pfmm_probe_fma_rate(1 if fp64 else 0, ctypes.byref(v), _stream(stream)))
    return v.value


def pfmm_default_solve_opts() -> pfmm_solve_opts:
    o = pfmm_solve_opts()
    _check(lib().pfmm_default_solve_opts(ctypes.byref(o)))
    return o


def pfmm_solve(h, formulation: int, g, x, nrhs: int, opts: pfmm_solve_opts | None = None, stream=None,
               allow_not_converged: bool = False) -> dict:
    """Solve V_h x = b (b from g by the chosen formulation); returns the solve info as a dict."""
    info = pfmm_solve_info()
    if opts is None:
        opts = pfmm_default_solve_opts()
    rc = lib().pfmm_solve(h, int(formulation), _ptr(g), _ptr(x), int(nrhs), ctypes.byref(opts), ctypes.byref(info),
                          _stream(stream))
    if not (rc == -6 and allow_not_converged):
        _check(rc)
    return dict(iterations=info.iterations, outer=info.outer, rel_res=info.rel_res, seconds=info.seconds,
                converged=rc == PFMM_OK, recorded=info.recorded, precond_off=info.precond_off)


def _mesh_struct(vertices, triangles, T, n_steps, alpha):
    V = np.ascontiguousarray(vertices, dtype=np.float64)
    Tr = np.ascontiguousarray(triangles, dtype=np.int32)
    m = pfmm_mesh(V.shape[0], Tr.shape[0], V.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                  Tr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), float(T), int(n_steps), float(alpha))
    m._keep = (V, Tr)
    return m


def pfmm_autotune_params(vertices, triangles, T, n_steps, alpha=1.0, base: pfmm_params | None = None, tol=1e-6,
                         m_lo=4, m_hi=8) -> pfmm_params:
    m = _mesh_struct(vertices, triangles, T, n_steps, alpha)
    out = pfmm_params()
    _check(lib().pfmm_autotune_params(ctypes.byref(m), ctypes.byref(base or pfmm_default_params()), float(tol),
                                      int(m_lo), int(m_hi), ctypes.byref(out)))
    return out


class Batch:
    """A batch of independent problems applied through one captured CUDA graph."""

    def __init__(self, problems, tune_engines=False, stream=None):
        """problems: list of (vertices, triangles, T, n_steps, alpha, pfmm_params)."""
        n = len(problems)
        meshes = (pfmm_mesh * n)()
        params = (pfmm_params * n)()
        self._keep = []
        for i, (V, Tr, T, Et, alpha, prm) in enumerate(problems):
            m = _mesh_struct(V, Tr, T, Et, alpha)
            self._keep.append(m._keep)
            meshes[i] = m
            params[i] = prm
        self.b = ctypes.c_void_p()
        _check(lib().pfmm_build_trees_batched(n, meshes, params, 1 if tune_engines else 0, _stream(stream),
                                              ctypes.byref(self.b)))
        self.n = n

    def handle(self, i):
        h = ctypes.c_void_p()
        _check(lib().pfmm_batch_handle(self.b, int(i), ctypes.byref(h)))
        return h

    def set_streams(self, n: int) -> None:
        _check(lib().pfmm_batch_set_streams(self.b, int(n)))

    def apply_V(self, ws, fs, stream=None):
        n = self.n
        wp = (ctypes.c_void_p * n)(*[_ptr(w) for w in ws])
        fp = (ctypes.c_void_p * n)(*[_ptr(f) for f in fs])
        nr = (ctypes.c_int32 * n)(*[int(w.shape[0]) for w in ws])
        _check(lib().pfmm_apply_V_batched(self.b, wp, fp, nr, _stream(stream)))

    def close(self):
        if self.b:
            lib().pfmm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pfmm_destroy(h):
    if h:
        lib().pfmm_destroy(h)


class Operator:
    """Convenience owner of a handle: V_h, K_h and M_h applies on torch CUDA tensors."""

    def __init__(self, vertices, triangles, T, n_steps, alpha=1.0, stream=None, **params):
        p = pfmm_default_params()
        for k, v in params.items():
            if not hasattr(p, k):
                raise TypeError(f"unknown parameter {k}")
            setattr(p, k, v)
        self.params = p
        self.nv = int(np.asarray(vertices).shape[0])
        self.nt = int(np.asarray(triangles).shape[0])
        self.n_steps = int(n_steps)
        self.h = pfmm_build_trees(vertices, triangles, T, n_steps, alpha, p, stream)

    def _out(self, x, ncol_in):
        import torch

        xx = x if x.dim() == 3 else x.unsqueeze(0)
        if xx.shape[1] != self.n_steps or xx.shape[2] != ncol_in:
            raise ValueError(f"expected [nrhs, {self.n_steps}, {ncol_in}], got {tuple(x.shape)}")
        xx = xx.contiguous()
        return xx, torch.empty((xx.shape[0], self.n_steps, self.nt), dtype=torch.float64, device=xx.device)

    def V(self, w, parts=PFMM_PART_ALL, stream=None):
        ww, f = self._out(w, self.nt)
        pfmm_apply_parts(self.h, 0, ww, f, ww.shape[0], parts, stream)
        return f if w.dim() == 3 else f[0]

    def K(self, g, parts=PFMM_PART_ALL, stream=None):
        gg, f = self._out(g, self.nv)
        pfmm_apply_parts(self.h, 1, gg, f, gg.shape[0], parts, stream)
        return f if g.dim() == 3 else f[0]

    def M(self, g, stream=None):
        gg, f = self._out(g, self.nv)
        pfmm_apply_M(self.h, gg, f, gg.shape[0], stream)
        return f if g.dim() == 3 else f[0]

    def info(self):
        return pfmm_get_info(self.h)

    def close(self):
        if self.h:
            pfmm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GeneralOperator:
    """V_h on general (non-uniform) time steps t_steps[0] = 0 < ... < t_steps[E_t] = T (pfmm_gen_*):
    the FMM on the general tree of Alg. 1 with early leaves; n_max is Alg. 1's element bound."""

    def __init__(self, vertices, triangles, t_steps, n_max, alpha=1.0, stream=None, **params):
        p = pfmm_default_params()
        for k, v in params.items():
            if not hasattr(p, k):
                raise TypeError(f"unknown parameter {k}")
            setattr(p, k, v)
        self.params = p
        self.h = None
        ts = np.ascontiguousarray(t_steps, dtype=np.float64)
        self.nt = int(np.asarray(triangles).shape[0])
        self.n_steps = ts.shape[0] - 1
        m = _mesh_struct(vertices, triangles, float(ts[-1]), self.n_steps, alpha)
        out = ctypes.c_void_p()
        _check(lib().pfmm_gen_create(ctypes.byref(m), ts.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     ctypes.byref(p), int(n_max), _stream(stream), ctypes.byref(out)))
        self.h = out.value

    def V(self, w, parts=PFMM_PART_ALL, stream=None):
        import torch

        ww = (w if w.dim() == 3 else w.unsqueeze(0)).contiguous()
        if ww.shape[1] != self.n_steps or ww.shape[2] != self.nt:
            raise ValueError(f"expected [nrhs, {self.n_steps}, {self.nt}], got {tuple(w.shape)}")
        f = torch.empty_like(ww)
        _check(lib().pfmm_gen_apply_V(self.h, _ptr(ww), _ptr(f), int(ww.shape[0]), int(parts), _stream(stream)))
        return f if w.dim() == 3 else f[0]

    def info(self) -> dict:
        i = pfmm_gen_info()
        _check(lib().pfmm_gen_get_info(self.h, ctypes.byref(i)))
        n = i.nlev
        out = {k: list(getattr(i, k)[:n]) for k in ("lx", "nbox", "nleaf", "nint", "ntr_far", "ntr_near", "st",
                                                     "pad")}
        out.update(nlev=n, n_m2l_pairs=i.n_m2l_pairs, n_near_blocks=i.n_near_blocks,
                   nearfield_entries=i.nearfield_entries, device_bytes=i.device_bytes)
        return out

    def boxes(self):
        """[nbox][8] rows (level, cell x, y, z, interval k, leaf, first step, end step)."""
        n = ctypes.c_int64()
        _check(lib().pfmm_gen_boxes(self.h, None, 0, ctypes.byref(n)))
        rows = np.zeros((max(n.value, 1), 8), np.int32)
        _check(lib().pfmm_gen_boxes(self.h, rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), n.value,
                                    ctypes.byref(n)))
        return rows[:n.value]

    def close(self):
        if self.h:
            lib().pfmm_gen_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mpnn:
    """Learned right preconditioner of pfmm_solve (message passing over the triangle adjacency)."""

    def __init__(self, vertices, triangles, T, n_steps, alpha=1.0, width=64, layers=4, seed=0):
        m = _mesh_struct(vertices, triangles, T, n_steps, alpha)
        out = ctypes.c_void_p()
        _check(lib().pfmm_mpnn_create(ctypes.byref(m), int(width), int(layers), int(seed), ctypes.byref(out)))
        self.ptr = out.value
        self.nt = int(np.asarray(triangles).shape[0])
        self.n_steps = int(n_steps)

    def num_params(self) -> int:
        return int(lib().pfmm_mpnn_num_params(self.ptr))

    def get_params(self) -> np.ndarray:
        p = np.empty(self.num_params(), dtype=np.float32)
        _check(lib().pfmm_mpnn_get_params(self.ptr, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), p.size))
        return p

    def set_params(self, p) -> None:
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(lib().pfmm_mpnn_set_params(self.ptr, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), p.size))

    @property
    def output_scale(self) -> float:
        c = ctypes.c_float()
        _check(lib().pfmm_mpnn_get_output_scale(self.ptr, ctypes.byref(c)))
        return c.value

    @output_scale.setter
    def output_scale(self, c: float) -> None:
        _check(lib().pfmm_mpnn_set_output_scale(self.ptr, float(c)))

    def apply(self, v, z, stream=None) -> None:
        _check(lib().pfmm_mpnn_apply(self.ptr, _ptr(v), _ptr(z), int(v.shape[0]), _stream(stream)))

    def loss_grad(self, R, E, slices, handle=None, stream=None):
        """Loss and gradient; same-step form with a pFMM handle, error form (needs E) without."""
        sl = np.ascontiguousarray(slices, dtype=np.int32)
        loss = ctypes.c_float()
        g = np.empty(self.num_params(), dtype=np.float32)
        _check(lib().pfmm_mpnn_loss_grad(self.ptr, handle, _ptr(R), _ptr(E),
                                         sl.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), sl.size,
                                         ctypes.byref(loss), g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                         _stream(stream)))
        return loss.value, g

    def train(self, R, E, nvec, steps, batch_slices=32, lr=1e-3, seed=0, handle=None, stream=None) -> np.ndarray:
        hist = np.zeros(max(int(steps), 1), dtype=np.float32)
        _check(lib().pfmm_mpnn_train(self.ptr, handle, _ptr(R), _ptr(E), int(nvec), int(steps), int(batch_slices),
                                     float(lr), int(seed), hist.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                     _stream(stream)))
        return hist[:steps]

    def check(self) -> None:
        _check(lib().pfmm_mpnn_check(self.ptr))

    def compile(self, stream=None) -> None:
        """Assemble the per-step sparse operators the (linear) network equals; apply uses them."""
        _check(lib().pfmm_mpnn_compile(self.ptr, _stream(stream)))

    def close(self):
        if self.ptr:
            lib().pfmm_mpnn_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

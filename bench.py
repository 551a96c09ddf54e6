"""Benchmark: pFMM V_h matvec throughput (space-time DOF/s) on one GB300.

Workload (the single large problem): surface of the unit cube, 32 x 32 squares per face cut
into 12288 flat triangles, 256 uniform steps on [0, 1] (3,145,728 space-time DOFs), Chebyshev
degree 6 in space, Lagrange degree 4 in time, c_st = 1, temporal leaves of 2 steps.  A step is
one f = V_h w (the product every GMRES iteration applies), w ~ N(0,1) seeded.  The nearfield
blocks and tables are built before the timed region (assembly).  The headline value is the
FP64 product (the paper's precision); the mixed-precision product of the same workload is
reported beside it with its error against FP64 and against the CPU oracle.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed] [--impl ours|reference]

Prints one JSON line.  Under torchrun (N > 1) each rank runs its own replica of the problem
(the matvec does not shard on one box: replicas only), timing is the max over ranks and value
is the whole-job DOF/s.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pFMM matvec space-time DOF/s"
# DRAM bytes (read + write) per stored nearfield element of one FP64 residue-arithmetic nearfield
# launch (k_nf_apply_crt, form 1), from an ncu capture of the 3072-triangle x 256-step case
# (1.7167e9 B read + 1.18e7 B written over 50,331,648 stored elements); traffic grows with the
# stored elements, so a full launch's traffic is this times its element count
NF_CRT_DRAM_BYTES_PER_ELEMENT = (1.716715e9 + 1.1788e7) / 50331648
NF_CRT_TRAFFIC_SOURCE = ("ncu capture of 3072 tri x 256 steps (profiles/nf_crt_3072x256_fp64.md), scaled by the "
                         "stored elements")
N_A, ET, M_X, M_T, C_ST = 32, 256, 6, 4, 1.0


def _set_size(n_a, et):
    global N_A, ET
    N_A, ET = n_a, et


def _clock_sampler(stop, out):
    """nvidia-smi in its own loop mode (a sample every 50 ms) while the timed region runs."""
    cmd = ["nvidia-smi", "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
           "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
           "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "50", "-i",
           os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or "0"]
    try:
        proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except OSError:
        return

    def reader():
        for line in proc.stdout:
            out.append(line.strip())

    t = threading.Thread(target=reader, daemon=True)
    t.start()
    stop.wait()
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
    t.join(timeout=2)


def _clocks_summary(samples):
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for s in samples:
        f = [x.strip() for x in s.split(",")]
        try:
            sm.append(float(f[0]))
            mx.append(float(f[1]))
        except (ValueError, IndexError):
            continue
        for n, v in zip(names, f[3:7]):
            if v.lower() in ("active", "1"):
                reasons.add(n)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_rows(V, T, Et, w, rows, nthreads=0, near=None):
    """The CPU oracle's V_h w on the sampled target rows: the nearfield rows as stored blocks
    (assembled before the timer, as the paper assembles before its GMRES iterations) times w over
    the nearfield offsets, plus the far field of the oracle's pFMM (Alg. 2: whole-mesh S2M and M2M,
    then M2L / L2L / L2T on the boxes of the sampled rows).  Returns the rows of f, the timings and
    the assembled blocks (for reuse)."""
    import oracle as O

    P_ = O.make_problem(V, T, 1.0, Et, m_t=M_T, m_x=M_X, c_st=C_ST)
    t0 = time.perf_counter()
    if near is None:
        near = O.assemble_V_rows(V, T, 1.0 / Et, rows, nd=4, nthreads=nthreads)
    t_asm = time.perf_counter() - t0
    t0 = time.perf_counter()
    fn = O.toeplitz_rows_apply(near, w, leaf_steps=2)
    t_near = time.perf_counter() - t0
    t0 = time.perf_counter()
    ff = O.pfmm_apply(P_, 0, w, targets=rows, parts=2, nthreads=nthreads)[:, rows]
    t_far = time.perf_counter() - t0
    return dict(f=fn + ff, t_assembly=t_asm, t_near=t_near, t_far=t_far), near


def _cpu_baseline(V, T, Et, w, every=64, nthreads=0):
    """cpu_baseline: the oracle's matvec (stored nearfield rows, pFMM far field) on every
    `every`-th target triangle (all Et steps) of the workload, in space-time DOF/s of the sampled
    rows; plus the far field's fixed whole-mesh cost (one target row) for context."""
    import oracle as O

    rows = np.arange(0, T.shape[0], every, dtype=np.int32)
    r, near = _oracle_rows(V, T, Et, w, rows, nthreads)
    P_ = O.make_problem(V, T, 1.0, Et, m_t=M_T, m_x=M_X, c_st=C_ST)
    t0 = time.perf_counter()
    O.pfmm_apply(P_, 0, w, targets=rows[:1], parts=2, nthreads=nthreads)
    t_fixed = time.perf_counter() - t0
    t = r["t_near"] + r["t_far"]
    cores = nthreads if nthreads > 0 else _host_cores()
    cb = dict(value=len(rows) * Et / t, unit="space-time DOF/s", cores=cores, kind="oracle",
              sample=f"V_h w on every {every}th target triangle ({len(rows)} rows x {Et} steps): nearfield rows as "
                     f"stored blocks (assembled outside the timer, {r['t_assembly']:.1f} s) x w, plus the oracle pFMM "
                     f"far field of those rows; {t:.1f} s",
              near_s=r["t_near"], far_s=r["t_far"], far_fixed_one_row_s=t_fixed, assembly_s=r["t_assembly"])
    return cb, rows, r["f"]


def _dense_rows_error(V, T, Et, w, outs, n_rows=8, nthreads=0):
    """Error of each GPU output against the dense Galerkin V_h (every step offset, no FMM
    approximation) on n_rows sampled target triangles (the oracle's plain definition, Section 2)."""
    import oracle as O
    from paper_2106_15911_gb300.inputs import sample_triangles

    rows = sample_triangles(T.shape[0], n_rows, seed=64)
    blocks = np.concatenate([O.assemble_V_rows(V, T, 1.0 / Et, rows, d0=d0, nd=min(64, Et - d0), nthreads=nthreads)
                             for d0 in range(0, Et, 64)])
    ref = O.toeplitz_rows_apply(blocks, w)
    den = np.max(np.abs(ref))
    return {k: float(np.max(np.abs(v[:, rows] - ref)) / den) for k, v in outs.items()}, len(rows)


# FP32 operations of one double-FP32 multiply-add (FMA two-product, two-sum, renormalisation):
# the FP64 mode's FMM passes reach at most the FP32 rate divided by this
DF64_FP32_OPS_PER_MAC = 15


def phase_rooflines(phases, info, es, nt, Et, mx, mt, peaks, arith=None):
    """Algorithmic work per apply of every phase, the rate it achieved in its measured phase time
    and the fraction of the peak of the unit it runs on.  S2M / L2T: 2 E_t E_x n_kappa + 4 (leaves)
    n_a n_kappa flops; M2L: the separable passes' flops reported by the library (info m2l_flops);
    nearfield: 2 sum_t |D(t)| nnz(A_d) flops on the stored elements.  arith: "fp32" (mixed mode),
    "df64" (FP64 mode: passes in double-FP32 on the FP32 pipe, peak = FP32 rate /
    DF64_FP32_OPS_PER_MAC; nearfield as residue products on the tensor cores where the handle
    has them, 32 B per stored element) or "fp64" (native FP64 on the FP64 pipe); default from es.
    peaks: hbm_gbs, fp64_tflops, fp32_tflops, fp16_tflops."""
    from math import comb

    arith = arith or ("fp64" if es == 8 else "fp32")
    nk, na = comb(mx + 3, 3), mt + 1
    p = info["p"]
    nleaf = info["nbox"][p] * (Et // 2)
    dof = nt * Et
    if arith == "df64":
        fma, fsrc = peaks["fp32_tflops"] / DF64_FP32_OPS_PER_MAC, "FP32 FMA rate / %d (double-FP32)" % DF64_FP32_OPS_PER_MAC
    elif arith == "fp64":
        fma, fsrc = peaks["fp64_tflops"], "FP64 FMA rate"
    else:
        fma, fsrc = peaks["fp32_tflops"], "FP32 FMA rate"
    out = {}

    def put(name, flops, byts, ms, fpeak, src):
        if not ms or ms <= 0:
            return
        d = {"ms": ms, "flops": flops, "bytes": byts, "tflops": flops / (ms * 1e-3) / 1e12,
             "gbs": byts / (ms * 1e-3) / 1e9}
        d["frac_fp"] = d["tflops"] / fpeak
        d["frac_hbm"] = d["gbs"] / peaks["hbm_gbs"]
        d["bound"] = "fp" if d["frac_fp"] >= d["frac_hbm"] else "hbm"
        d["fp_peak_tflops"], d["fp_peak"] = fpeak, src
        out[name] = d

    s2m_f = 2.0 * Et * nt * nk + 2.0 * nleaf * 2 * na * nk
    put("s2m", s2m_f, es * dof + es * nt * nk + es * nleaf * na * nk, phases.get("s2m"), fma, fsrc)
    put("l2t", s2m_f, 16.0 * dof + es * nt * nk + es * nleaf * na * nk, phases.get("l2t"), fma, fsrc)
    if p >= 2:
        put("m2l", info["m2l_flops"],
            2.0 * es * sum(info["nbox"][l] * 2 ** l for l in range(2, p + 1)) * na * nk, phases.get("m2l"), fma, fsrc)
    nel = info["nearfield_v_elements"]
    nf_flops = 2.0 * (nel / 4) * (Et // 2) * 7  # 2 sum_t |D(t)| nnz(A_d): |D| = 3, 4 on the two steps
    tc = bool(info.get("nf_tensor_cores", 0) & 1)
    if tc and arith == "fp32":  # scaled FP16 hi / lo parts: 4 B per element, 3 FP16 products
        put("nearfield", nf_flops, nel * 4 + 16.0 * dof, phases.get("nearfield"), peaks["fp16_tflops"] / 3,
            "FP16 tensor peak / 3 (hi / lo products)")
    elif tc and arith == "df64":  # residues modulo 16 primes: 32 B per element, 16 FP16 products
        put("nearfield", nf_flops, nel * 32 + 48.0 * dof, phases.get("nearfield"), peaks["fp16_tflops"] / 16,
            "FP16 tensor peak / 16 (residue products)")
    else:
        put("nearfield", nf_flops, nel * es + 16.0 * dof, phases.get("nearfield"), peaks["fp64_tflops"] if es == 8
            else peaks["fp32_tflops"], "FP64 FMA rate" if es == 8 else "FP32 FMA rate")
    return out


def _solve_comparison(dev, n_train=256, n_test=32):
    """Time to 1e-8 relative residual (Eq. 02:linear:system, direct formulation) on the
    3072-triangle x 128-step cube, averaged over held-out data sets: plain FP64 FGMRES(50),
    GMRES-IR (mixed-precision inner FGMRES, FP64 residuals), and GMRES-IR with the learned
    preconditioner.  The network (width 64, 4 layers) is trained on residual slices that mixed
    FGMRES runs record on n_train data sets (one heat source each, rng seeds 4 + k), in the
    same-step form; the held-out sets use seeds 4 + n_train + k."""
    import numpy as np
    import torch

    from paper_2106_15911_gb300 import pfmm as P
    from paper_2106_15911_gb300.inputs import cube_mesh, heat_source_datum, shell_sources

    V, T = cube_mesh(16)
    Et, nt = 128, T.shape[0]
    kw = dict(m_t=4, m_x=6, c_st=1.0)
    op64 = P.Operator(V, T, 1.0, Et, **kw)
    opm = P.Operator(V, T, 1.0, Et, precision=P.PFMM_MIXED, **kw)

    def datum(seed):
        return torch.tensor(heat_source_datum(V, 1.0, Et, shell_sources(1, seed=seed))[None], device=dev)

    per_set = 20
    R = torch.empty((n_train * per_set, Et, nt), dtype=torch.float64, device=dev)
    x = torch.empty((1, Et, nt), dtype=torch.float64, device=dev)
    used, t0 = 0, time.perf_counter()
    for k in range(n_train):
        o = P.pfmm_default_solve_opts()
        o.tol, o.rec_r, o.rec_cap, o.rec_every = 1e-6, R[used].data_ptr(), per_set, 5
        used += P.pfmm_solve(opm.h, P.PFMM_DIRECT, datum(4 + k), x, 1, o, allow_not_converged=True)["recorded"]
    t_gen = time.perf_counter() - t0
    net = P.Mpnn(V, T, 1.0, Et, width=64, layers=4, seed=7)
    t0 = time.perf_counter()
    hist = net.train(R, None, used, steps=1500, batch_slices=32, lr=3e-3, seed=8, handle=opm.h)
    t_train = time.perf_counter() - t0
    del R
    zz = torch.empty_like(x)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def t_net():
        net.apply(x, zz)
        e0.record()
        for _ in range(10):
            net.apply(x, zz)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 10

    t_apply = t_net()  # the network's layer kernels
    t0 = time.perf_counter()
    net.compile()  # its per-step sparse operators, used by the solves below
    t_compile = time.perf_counter() - t0
    t_apply_c = t_net()
    arms = {"fp64_fgmres": [], "mixed_gmres_ir": [], "mixed_gmres_ir_learned": []}
    worst_diff = 0.0
    for k in range(n_test):
        g = datum(4 + n_train + k)
        arms["fp64_fgmres"].append(P.pfmm_solve(op64.h, P.PFMM_DIRECT, g, x, 1))
        x64 = x.clone()
        o = P.pfmm_default_solve_opts()
        o.refine = op64.h
        arms["mixed_gmres_ir"].append(P.pfmm_solve(opm.h, P.PFMM_DIRECT, g, x, 1, o))
        o.precond = net.ptr
        arms["mixed_gmres_ir_learned"].append(P.pfmm_solve(opm.h, P.PFMM_DIRECT, g, x, 1, o))
        worst_diff = max(worst_diff, float((x - x64).abs().max() / x64.abs().max()))
    net.close()
    op64.close()
    opm.close()

    def summ(rs):
        return {"mean_iterations": float(np.mean([r["iterations"] for r in rs])),
                "mean_seconds": float(np.mean([r["seconds"] for r in rs])),
                "worst_rel_res": float(max(r["rel_res"] for r in rs)), "all_converged": all(r["converged"] for r in rs),
                "precond_dropped": int(sum(r["precond_off"] for r in rs))}

    out = {k: summ(v) for k, v in arms.items()}
    return {"workload": f"cube 16x16 faces ({nt} tri) x {Et} steps, direct formulation, tol 1e-8, "
                        f"{n_test} held-out heat-source data sets",
            "training": {"data_sets": n_train, "recorded_residuals": used, "record_s": t_gen, "train_s": t_train,
                         "steps": 1500, "loss_first": float(hist[:10].mean()), "loss_last": float(hist[-50:].mean()),
                         "network": "width 64, 4 layers, BF16 weights, tcgen05 layers", "apply_ms": t_apply,
                         "compile_s": t_compile, "compiled_apply_ms": t_apply_c},
            **out,
            "speedup_learned_vs_fp64": out["fp64_fgmres"]["mean_seconds"] / out["mixed_gmres_ir_learned"]["mean_seconds"],
            "speedup_learned_vs_mixed": out["mixed_gmres_ir"]["mean_seconds"] / out["mixed_gmres_ir_learned"]["mean_seconds"],
            "worst_solution_rel_diff_vs_fp64": worst_diff}


def _batch_comparison(dev, n_problems, seed=3, tol=3e-3):
    """Ragged batch of independent problems (cube and cube-sphere surfaces alternating, triangle
    counts drawn from {768, 1536, 3072, 6144, 12288}, 32..256 steps, 1..8 right-hand sides,
    mixed precision, degree m_x in [4, 8] chosen by the autotuner for a farfield truncation
    estimate of `tol`, nearfield engine chosen by timing): replays of the captured CUDA graph
    with 16, 4 and 1 streams vs the same applies issued one after the other on one stream."""
    import numpy as np
    import torch

    from paper_2106_15911_gb300 import pfmm as P
    from paper_2106_15911_gb300.inputs import cube_mesh, cube_sphere_mesh, random_density

    rng = np.random.default_rng(seed)
    probs, dofs = [], 0
    for i in range(n_problems):
        n_a, split = [(8, "diag"), (8, "cross"), (16, "diag"), (16, "cross"), (32, "diag")][int(rng.integers(0, 5))]
        V, T = (cube_mesh if i % 2 == 0 else cube_sphere_mesh)(n_a, split)
        Et = int(rng.choice([32, 64, 128, 256]))
        nr = int(rng.integers(1, 9))
        prm = P.pfmm_default_params()
        prm.precision = P.PFMM_MIXED
        prm = P.pfmm_autotune_params(V, T, 1.0, Et, base=prm, tol=tol, m_lo=4, m_hi=8)
        probs.append((V, T, 1.0, Et, 1.0, prm, nr))
        dofs += T.shape[0] * Et * nr
    tb = time.perf_counter()
    B = P.Batch([p[:6] for p in probs], tune_engines=True)
    t_build = time.perf_counter() - tb
    ws = [torch.tensor(random_density(p[3], p[1].shape[0], p[6], seed=100 + i), device=dev) for i, p in enumerate(probs)]
    fs = [torch.empty_like(w) for w in ws]
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=5):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    graph_ms = {}
    for ns in (16, 4, 1):
        B.set_streams(ns)
        graph_ms[ns] = timed(lambda: B.apply_V(ws, fs))
    hs = [B.handle(i) for i in range(len(probs))]

    def seq():
        for h, w, f in zip(hs, ws, fs):
            P.pfmm_apply_V(h, w, f, w.shape[0], stream)

    t_seq = timed(seq)

    # where the batch's time goes: every problem's apply alone, with its phases (CUDA events
    # between the phases), summed by phase and by degree
    by_phase = dict.fromkeys(P.PHASES, 0.0)
    by_mx, per_problem = {}, []
    for i, (h, w, f) in enumerate(zip(hs, ws, fs)):
        P.pfmm_apply_V(h, w, f, w.shape[0], stream)
        P.pfmm_phase_times(h)
        P.pfmm_set_profiling(h, True)
        for _ in range(3):
            P.pfmm_apply_V(h, w, f, w.shape[0], stream)
        torch.cuda.synchronize()
        ph, n = P.pfmm_phase_times(h)
        P.pfmm_set_profiling(h, False)
        ms = sum(ph.values()) / max(n, 1)
        for k in by_phase:
            by_phase[k] += ph[k] / max(n, 1)
        m = str(int(probs[i][5].m_x))
        by_mx[m] = by_mx.get(m, 0.0) + ms
        per_problem.append((ms, probs[i][1].shape[0], probs[i][3], probs[i][6], int(probs[i][5].m_x)))
    B.close()
    best = min(graph_ms.values())
    mx = [int(p[5].m_x) for p in probs]
    per_problem.sort(reverse=True)
    return {"workload": f"{n_problems} problems, 768..12288 triangles, 32..256 steps, 1..8 rhs, mixed, "
                        f"autotuned m_x (truncation estimate {tol:g})",
            "space_time_dofs": dofs, "graph_ms_by_streams": graph_ms, "sequential_ms": t_seq,
            "dofs_per_s": dofs / (best * 1e-3), "build_s": t_build,
            "m_x_histogram": {str(m): mx.count(m) for m in sorted(set(mx))},
            "alone_ms_sum": sum(p[0] for p in per_problem), "alone_ms_by_phase": by_phase,
            "alone_ms_by_m_x": by_mx,
            "alone_top8": [{"ms": p[0], "triangles": p[1], "steps": p[2], "rhs": p[3], "m_x": p[4]}
                           for p in per_problem[:8]]}


def _config5(dev, n_rhs=4, n_record=2, tol=1e-6, solve=True):
    """Large combined run: cube-sphere 49152 triangles x 1024 steps (50.3M space-time DOF),
    m_x 6, m_t 4, mixed precision with the stored (dense-column, tensor-core) nearfield, learned
    preconditioner retrained at this size on residuals recorded by mixed FGMRES(30) runs, then
    n_rhs heat-source data sets solved with FGMRES(30) + the network (and one without it) to
    `tol` in the mixed operator; device memory is sampled after every stage (cap 180 GB).
    solve=False: the build and the matvecs only (1 and n_rhs right-hand sides, phase times of one
    single-rhs apply)."""
    import torch

    from paper_2106_15911_gb300 import pfmm as P
    from paper_2106_15911_gb300.inputs import cube_sphere_mesh, heat_source_datum, shell_sources

    V, T = cube_sphere_mesh(64)
    Et, nt = 1024, T.shape[0]
    free0, total = torch.cuda.mem_get_info()
    peak = [0.0]

    def track():
        peak[0] = max(peak[0], (free0 - torch.cuda.mem_get_info()[0]) / 1e9)

    t0 = time.perf_counter()
    opm = P.Operator(V, T, 1.0, Et, m_t=4, m_x=6, c_st=1.0, precision=P.PFMM_MIXED)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    info = opm.info()
    track()
    w = torch.randn((n_rhs, Et, nt), dtype=torch.float64, device=dev)
    f = torch.empty_like(w)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    mv_ms = {}
    for nr in (1, n_rhs):
        P.pfmm_apply_V(opm.h, w, f, nr, None)
        e0.record()
        P.pfmm_apply_V(opm.h, w, f, nr, None)
        e1.record()
        torch.cuda.synchronize()
        mv_ms[str(nr)] = e0.elapsed_time(e1)
    P.pfmm_set_profiling(opm.h, True)
    P.pfmm_apply_V(opm.h, w, f, 1, None)
    torch.cuda.synchronize()
    ph, nph = P.pfmm_phase_times(opm.h)
    P.pfmm_set_profiling(opm.h, False)
    phases = {k: v / max(nph, 1) for k, v in ph.items()}
    track()
    del w, f
    head = {"workload": f"cube-sphere {nt} tri x {Et} steps ({nt * Et} DOF), m_x 6, m_t 4, mixed, stored nearfield",
            "build_s": build_s, "nearfield_GB": info["nearfield_bytes"] / 1e9, "nf_tensor_cores": info["nf_tensor_cores"],
            "matvec_ms_nrhs": mv_ms, "matvec_dofs_per_s": n_rhs * nt * Et / (mv_ms[str(n_rhs)] * 1e-3),
            "phases_ms_1rhs": phases}
    if not solve:
        opm.close()
        return dict(head, peak_device_GB=peak[0], device_total_GB=total / 1e9, cap_GB=180)

    def datum(seed):
        return torch.tensor(heat_source_datum(V, 1.0, Et, shell_sources(1, seed=seed))[None], device=dev)

    per = 8
    R = torch.empty((n_record * per, Et, nt), dtype=torch.float64, device=dev)
    x = torch.empty((1, Et, nt), dtype=torch.float64, device=dev)
    used, t0 = 0, time.perf_counter()
    for k in range(n_record):
        o = P.pfmm_default_solve_opts()
        o.tol, o.restart, o.rec_r, o.rec_cap, o.rec_every = tol, 30, R[used].data_ptr(), per, 4
        used += P.pfmm_solve(opm.h, P.PFMM_DIRECT, datum(4 + k), x, 1, o, allow_not_converged=True)["recorded"]
        track()
    rec_s = time.perf_counter() - t0
    net = P.Mpnn(V, T, 1.0, Et, width=64, layers=4, seed=7)
    t0 = time.perf_counter()
    hist = net.train(R, None, used, steps=1000, batch_slices=16, lr=3e-3, seed=8, handle=opm.h)
    train_s = time.perf_counter() - t0
    track()
    del R
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    net.compile()
    compile_s = time.perf_counter() - t0
    track()
    torch.cuda.empty_cache()
    solves = []
    for k in range(n_rhs):
        o = P.pfmm_default_solve_opts()
        o.tol, o.restart, o.precond = tol, 30, net.ptr
        solves.append(P.pfmm_solve(opm.h, P.PFMM_DIRECT, datum(5000 + k), x, 1, o, allow_not_converged=True))
        track()
    o = P.pfmm_default_solve_opts()
    o.tol, o.restart = tol, 30
    plain = P.pfmm_solve(opm.h, P.PFMM_DIRECT, datum(5000), x, 1, o, allow_not_converged=True)
    track()
    net.close()
    opm.close()
    return dict(head, **{
            "record": {"data_sets": n_record, "residuals": used, "seconds": rec_s},
            "train": {"steps": 1000, "seconds": train_s, "loss_first": float(hist[:10].mean()),
                      "loss_last": float(hist[-50:].mean()), "compile_s": compile_s},
            "solve_tol": tol, "learned": solves, "plain_first_rhs": plain,
            "peak_device_GB": peak[0], "device_total_GB": total / 1e9, "cap_GB": 180})


def _paper_scale(dev, steps=5, dense_rows=4):
    """The parameter set of the paper's large distributed run (Section 5, Tab. mpi: m_x = 12,
    m_t = 4, c_st = 4.1, n_tr = 2) on its 12288 x 1024 shape: the unit-cube surface, 32 x 32
    squares per face, 1024 steps on [0, 1] (12.6M space-time DOF).  Mixed and FP64 V_h matvecs
    (build time, phases, throughput) and the truncation error of both against the dense Galerkin
    V_h of the oracle on sampled rows (the paper quotes 1.5 s per GMRES iteration on 256 CPU nodes
    for this shape, context only)."""
    import torch

    from paper_2106_15911_gb300 import pfmm as P
    from paper_2106_15911_gb300.inputs import cube_mesh, random_density

    V, T = cube_mesh(32)
    Et, nt = 1024, T.shape[0]
    kw = dict(m_t=4, m_x=12, c_st=4.1, n_tr=2)
    w = torch.tensor(random_density(Et, nt, 1, seed=4100), device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out, res = {}, {}
    for name, prec in (("mixed", P.PFMM_MIXED), ("fp64", P.PFMM_FP64)):
        t0 = time.perf_counter()
        op = P.Operator(V, T, 1.0, Et, precision=prec, **kw)
        torch.cuda.synchronize()
        build_s = time.perf_counter() - t0
        info = op.info()
        f = torch.empty_like(w)
        for _ in range(2):
            P.pfmm_apply_V(op.h, w, f, 1, None)
        e0.record()
        for _ in range(steps):
            P.pfmm_apply_V(op.h, w, f, 1, None)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        P.pfmm_set_profiling(op.h, True)
        P.pfmm_apply_V(op.h, w, f, 1, None)
        ph, n = P.pfmm_phase_times(op.h)
        P.pfmm_set_profiling(op.h, False)
        res[name] = f[0].cpu().numpy()
        out[name] = {"build_s": build_s, "ms_per_matvec": ms, "dofs_per_s": nt * Et / (ms * 1e-3),
                     "phases_ms": {k: v / max(n, 1) for k, v in ph.items()}, "tree_lx": info["lx"],
                     "nearfield_GB": info["nearfield_bytes"] / 1e9, "nf_tensor_cores": info["nf_tensor_cores"],
                     "nf_dense_columns": info["nf_dense_columns"], "m2l_engine": info["m2l_engine"],
                     "m2l_gflop": info["m2l_flops"] / 1e9}
        op.close()
        torch.cuda.empty_cache()
    rel = float(np.max(np.abs(res["mixed"] - res["fp64"])) / np.max(np.abs(res["fp64"])))
    dense = None
    if dense_rows > 0:
        dense, nr = _dense_rows_error(V, T, Et, w[0].cpu().numpy(), res, dense_rows)
        dense["rows"] = nr
    return {"workload": f"cube 32x32 faces ({nt} tri) x {Et} steps, m_x 12, m_t 4, c_st 4.1, n_tr 2 (Section 5 "
                        f"parameters)", **out, "mixed_vs_fp64_rel_maxnorm": rel, "vs_dense_oracle": dense,
            "paper": "1.5 s per GMRES iteration on 256 Salomon nodes (Tab. mpi), CPU cluster, context only"}


def _general_steps(dev, n_a=8, Et=64, n_max=200, steps=10, oracle_rows=6):
    """General (non-uniform) time steps (pfmm_gen_*: the tree of Alg. 1 with early leaves, no
    Toeplitz structure): cube with n_a x n_a squares per face, Et graded steps t_j = (j / Et)^1.5 on
    [0, 1], n_max = 200, m_t 4, m_x 6.  V_h matvec throughput (CUDA events, the stored step-pair
    nearfield of several GB is larger than L2), the nearfield and far-field parts alone, the
    nearfield apply's HBM roofline (8 bytes per stored entry), and parity with the oracle's pFMM on
    the same tree: far field on every row, nearfield on `oracle_rows` sampled triangles."""
    import torch

    import oracle as O
    from paper_2106_15911_gb300 import pfmm as P
    from paper_2106_15911_gb300.inputs import cube_mesh, random_density

    V, T = cube_mesh(n_a)
    nt = T.shape[0]
    ts = np.linspace(0.0, 1.0, Et + 1) ** 1.5
    kw = dict(m_t=4, m_x=6)
    t0 = time.perf_counter()
    op = P.GeneralOperator(V, T, ts, n_max, **kw)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    info = op.info()
    w = torch.tensor(random_density(Et, nt, 1, seed=2106)[0], device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = {}
    for name, parts in (("all", P.PFMM_PART_ALL), ("near", P.PFMM_PART_NEAR), ("far", P.PFMM_PART_FAR)):
        for _ in range(3):
            f = op.V(w, parts=parts)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            f = op.V(w, parts=parts)
        e1.record()
        torch.cuda.synchronize()
        ms[name] = e0.elapsed_time(e1) / steps
    f = op.V(w).cpu().numpy()
    near = op.V(w, parts=P.PFMM_PART_NEAR).cpu().numpy()
    peaks = _peaks(P, torch.cuda.current_stream())
    nf_bytes = 8.0 * info["nearfield_entries"] + 16.0 * nt * Et
    gbs = nf_bytes / (ms["near"] * 1e-3) / 1e9
    Pr = O.make_general_problem(V, T, ts, **kw)
    wn = w.cpu().numpy()
    far_ref = O.gen_pfmm_apply(Pr, n_max, wn, parts=P.PFMM_PART_FAR)
    rows = np.linspace(0, nt - 1, oracle_rows).astype(np.int32)
    near_ref = O.gen_pfmm_apply(Pr, n_max, wn, targets=rows, parts=P.PFMM_PART_NEAR)[:, rows]
    rel_far = float(np.max(np.abs((f - near) - far_ref)) / np.max(np.abs(far_ref)))
    rel_near = float(np.max(np.abs(near[:, rows] - near_ref)) / np.max(np.abs(near_ref)))
    op.close()
    return {"workload": f"cube {n_a}x{n_a} faces ({nt} tri) x {Et} graded steps t_j = (j/{Et})^1.5, n_max {n_max}, "
                        f"m_t 4, m_x 6, FP64", "dof": nt * Et, "build_s": build_s,
            "ms_per_matvec": ms["all"], "dofs_per_s": nt * Et / (ms["all"] * 1e-3),
            "ms_nearfield_only": ms["near"], "ms_farfield_only": ms["far"],
            "tree": {k: info[k] for k in ("nlev", "lx", "nbox", "nleaf", "nint")},
            "n_m2l_pairs": info["n_m2l_pairs"], "nearfield_entries": info["nearfield_entries"],
            "nearfield_GB": 8e-9 * info["nearfield_entries"],
            "roofline_nearfield": {"kernel": "k_gen_nf_apply", "bound": "hbm", "achieved": gbs,
                                   "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
                                   "bytes_per_launch": nf_bytes, "timing": "nearfield-only apply (permutes included)"},
            "parity_vs_oracle": {"far_all_rows": rel_far, "near_rows": int(rows.shape[0]), "near": rel_near}}


def _profile_case(dev, case):
    """Small cases for ncu captures: the learned preconditioner's layers (`mpnn`), its compiled
    form (`mpnn_compiled`), the on-the-fly nearfield (`otf`), the slab M2L of 8^3 grids
    (`m2l_slab`), the FP64 residue-arithmetic nearfield (`crt`, 3072 triangles x 256 steps), the
    general-step product (`general`, 768 triangles x 64 graded steps, as bench --general), the FP64
    far field (`passes`: S2M, M2M, M2L, L2L, L2T in double-FP32, 3072 triangles x 256 steps).  3072-triangle cube; 128 steps
    (network) or 32 steps (on-the-fly); 1728-triangle cube x 32 steps with an 8^3 leaf grid
    (c_st 0.1, interaction radius 7) for the slab M2L, far field only."""
    import numpy as np
    import torch

    from paper_2106_15911_gb300 import pfmm as P
    from paper_2106_15911_gb300.inputs import cube_mesh

    V, T = cube_mesh(16)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if case in ("mpnn", "mpnn_compiled"):
        Et = 128
        net = P.Mpnn(V, T, 1.0, Et, width=64, layers=4, seed=1)
        net.set_params((np.random.default_rng(0).standard_normal(net.num_params()) * 0.1).astype(np.float32))
        net.output_scale = 1.0
        if case == "mpnn_compiled":
            net.compile()
        v = torch.randn((1, Et, len(T)), dtype=torch.float64, device=dev)
        z = torch.empty_like(v)
        run = lambda: net.apply(v, z)  # noqa: E731
    elif case == "crt":
        Et = 256
        op = P.Operator(V, T, 1.0, Et, m_t=4, m_x=6, c_st=1.0, precision=P.PFMM_FP64)
        w = torch.randn((1, Et, len(T)), dtype=torch.float64, device=dev)
        run = lambda: op.V(w, parts=P.PFMM_PART_NEAR)  # noqa: E731
    elif case == "passes":
        Et = 256
        op = P.Operator(V, T, 1.0, Et, m_t=4, m_x=6, c_st=1.0, precision=P.PFMM_FP64)
        w = torch.randn((1, Et, len(T)), dtype=torch.float64, device=dev)
        run = lambda: op.V(w, parts=P.PFMM_PART_FAR)  # noqa: E731
    elif case == "general":
        V, T = cube_mesh(8)
        Et = 64
        op = P.GeneralOperator(V, T, np.linspace(0.0, 1.0, Et + 1) ** 1.5, 200, m_t=4, m_x=6)
        w = torch.randn((1, Et, len(T)), dtype=torch.float64, device=dev)
        run = lambda: op.V(w)  # noqa: E731
    elif case == "m2l_slab":
        V, T = cube_mesh(12)
        Et = 32
        op = P.Operator(V, T, 1.0, Et, m_t=4, m_x=6, c_st=0.1, precision=P.PFMM_MIXED)
        w = torch.randn((1, Et, len(T)), dtype=torch.float64, device=dev)
        run = lambda: op.V(w, parts=P.PFMM_PART_FAR)  # noqa: E731
    else:
        Et = 32
        op = P.Operator(V, T, 1.0, Et, m_t=4, m_x=6, c_st=1.0, precision=P.PFMM_MIXED,
                        nearfield=P.PFMM_NEARFIELD_ONTHEFLY)
        w = torch.randn((1, Et, len(T)), dtype=torch.float64, device=dev)
        run = lambda: op.V(w, parts=P.PFMM_PART_NEAR)  # noqa: E731
    run()
    e0.record()
    for _ in range(2):
        run()
    e1.record()
    torch.cuda.synchronize()
    out = {"profile_case": case, "ms_per_call": e0.elapsed_time(e1) / 2}
    if case in ("crt", "m2l_slab", "otf", "passes"):
        info = op.info()
        out.update(nearfield_v_elements=info["nearfield_v_elements"], nf_form=info["nf_form"],
                   m2l_engine=info["m2l_engine"])
    return out


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest per-rank value (the slowest replica's time) on every rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replicas_throughput(units_per_rank: float, ms_step: float, world: int) -> float:
    """Whole-job throughput of `world` independent replicas: all ranks' units over the slowest
    rank's time (weak scaling, no data-path collective)."""
    return world * units_per_rank / (ms_step * 1e-3)


def reference_arm(args, rank, world):
    """The oracle (plain CPU FP64 pFMM of Alg. 2, nearfield rows stored) on the same workload:
    each step is V_h w on a bounded sample of target rows (every 384th triangle, 32 rows x 256
    steps), the nearfield rows assembled once before the steps."""
    if rank != 0:
        return 0
    from paper_2106_15911_gb300.inputs import cube_mesh, random_density

    V, T = cube_mesh(N_A)
    nt = T.shape[0]
    w = random_density(ET, nt, 1, seed=1234)[0]
    rows = np.arange(0, nt, 384, dtype=np.int32)
    near = None
    vals, tot = [], 0.0
    for i in range(args.warmup + args.steps):
        r, near = _oracle_rows(V, T, ET, w, rows, near=near)
        if i >= args.warmup:
            dt = r["t_near"] + r["t_far"]
            vals.append(len(rows) * ET / dt)
            tot += dt
    v = statistics.mean(vals)
    cb = {"value": v, "unit": "space-time DOF/s", "cores": _host_cores(), "kind": "oracle",
          "sample": f"V_h w on every 384th target triangle ({len(rows)} rows x {ET} steps) per step: stored "
                    f"nearfield rows x w plus the oracle pFMM far field of those rows"}
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "space-time DOF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config_dict(nt), "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "space-time DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _config_dict(nt, world=1):
    return {"workload": f"cube {N_A}x{N_A} faces ({nt} tri) x {ET} steps, V_h matvec", "dofs": nt * ET,
            "m_x": M_X, "m_t": M_T, "c_st": C_ST, "leaf_steps": 2, "n_tr": "derived (no truncation)",
            "l2": "flushed (256 MB write) between timed steps", "parallelism": f"replicas x{world}"}


def _peaks(P, stream):
    pk = {}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        pk = json.load(open(path))
    src = "of measured" if pk else "of fallback"
    return {"hbm_gbs": float(pk.get("hbm_gbs", 6800.0)), "fp16_tflops": float(pk.get("bf16_tflops", 1900.0)),
            "fp64_tflops": P.pfmm_probe_fma_rate(True, stream), "fp32_tflops": P.pfmm_probe_fma_rate(False, stream),
            "source": f"HBM and FP16 (= dense BF16 burst) {src} MEASURED_PEAKS.json; FP64 / FP32 FMA rates measured "
                      f"by pfmm_probe_fma_rate in this run"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="fp64",
                    help="precision of the headline value (the other one is reported beside it)")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--other-steps", type=int, default=10, help="timed steps of the other precision (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--dense-rows", type=int, default=8, help="rows of the dense-oracle error check (0: skip)")
    ap.add_argument("--no-solve", action="store_true", help="skip the solver comparison")
    ap.add_argument("--solve-sets", type=int, default=32, help="held-out data sets of the solver comparison")
    ap.add_argument("--config5", action="store_true", help="run only the 50M-DOF combined workload")
    ap.add_argument("--paper-scale", action="store_true",
                    help="run only the paper's large-run parameters (m_x 12, c_st 4.1, n_tr 2) on 12288 x 1024")
    ap.add_argument("--general", action="store_true",
                    help="run only the general (non-uniform) time-step FMM on 768 tri x 64 graded steps")
    ap.add_argument("--config5-matvec", action="store_true",
                    help="with --config5: the build and matvecs only (no recording, training or solves)")
    ap.add_argument("--profile-case", choices=["mpnn", "mpnn_compiled", "otf", "m2l_slab", "crt", "passes", "general"], default=None,
                    help="profiling only: run one small case of a kernel outside the matvec and exit")
    ap.add_argument("--batch", type=int, default=64, help="problems in the batch measurement (0: skip)")
    ap.add_argument("--n-a", type=int, default=N_A, help="profiling only: squares per cube face edge")
    ap.add_argument("--et", type=int, default=ET, help="profiling only: time steps")
    args = ap.parse_args()
    if (args.n_a, args.et) != (N_A, ET):
        _set_size(args.n_a, args.et)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import torch
    import torch.distributed as dist

    from paper_2106_15911_gb300 import pfmm as P
    from paper_2106_15911_gb300.inputs import cube_mesh, random_density

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.config5:
        if rank == 0:
            print(json.dumps({"config5": _config5(dev, solve=not args.config5_matvec)}), flush=True)
        return 0
    if args.profile_case:
        if rank == 0:
            print(json.dumps(_profile_case(dev, args.profile_case)), flush=True)
        return 0
    if args.paper_scale:
        if rank == 0:
            print(json.dumps({"paper_scale": _paper_scale(dev)}), flush=True)
        return 0
    if args.general:
        if rank == 0:
            print(json.dumps({"general_steps": _general_steps(dev)}), flush=True)
        return 0
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    V, T = cube_mesh(N_A)
    nt = T.shape[0]
    dof = nt * ET
    stream = torch.cuda.current_stream()
    head = P.PFMM_FP64 if args.precision == "fp64" else P.PFMM_MIXED
    other = P.PFMM_MIXED if head == P.PFMM_FP64 else P.PFMM_FP64

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def build(prec):
        t0 = time.perf_counter()
        o = P.Operator(V, T, 1.0, ET, m_t=M_T, m_x=M_X, c_st=C_ST, precision=prec)
        torch.cuda.synchronize()
        return o, time.perf_counter() - t0

    op, t_build = build(head)
    info = op.info()
    w = torch.tensor(random_density(ET, nt, 1, seed=1234 + rank), device=dev)
    f = torch.empty_like(w)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2

    def run_device_timed(steps, warm, opx, fx):
        P.pfmm_set_profiling(opx.h, False)
        for _ in range(warm):
            P.pfmm_apply_V(opx.h, w, fx, 1, stream)
        P.pfmm_nf_kernel_time(opx.h)
        P.pfmm_phase_times(opx.h)
        P.pfmm_set_profiling(opx.h, True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        barrier()
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(stream)
            P.pfmm_apply_V(opx.h, w, fx, 1, stream)
            ev[i][1].record(stream)
        barrier()
        ms = [a.elapsed_time(b) for a, b in ev]
        nf_ms, nf_n = P.pfmm_nf_kernel_time(opx.h)
        phases, n = P.pfmm_phase_times(opx.h)
        P.pfmm_set_profiling(opx.h, False)
        out = {k: v / max(n, 1) for k, v in phases.items()}
        out["nf_kernel"] = nf_ms / nf_n if nf_n else None
        return ms, out

    # ---- timed region (device), with live clock sampling
    stop, samples = threading.Event(), []
    th = threading.Thread(target=_clock_sampler, args=(stop, samples), daemon=True)
    th.start()
    time.sleep(0.3)  # the sampler's first line comes before the timed region
    n_before = len(samples)
    ms, phases = run_device_timed(args.steps, args.warmup, op, f)
    time.sleep(0.1)
    stop.set()
    th.join(timeout=10)
    samples = samples[max(0, n_before - 1):]  # the samples of (and bracketing) the timed region
    ms_step = max_over_ranks(statistics.mean(ms), world, dev)
    value = replicas_throughput(dof, ms_step, world)
    launches = P.pfmm_count_apply_kernels(op.h, 0, w, f, 1)

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timed region
    wh = torch.tensor(random_density(ET, nt, 1, seed=99 + rank)).pin_memory()
    fh = torch.empty_like(wh).pin_memory()
    wd, fd = torch.empty_like(w), torch.empty_like(f)
    for _ in range(args.warmup):
        wd.copy_(wh, non_blocking=True)
        P.pfmm_apply_V(op.h, wd, fd, 1, stream)
        fh.copy_(fd, non_blocking=True)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        wd.copy_(wh, non_blocking=True)
        P.pfmm_apply_V(op.h, wd, fd, 1, stream)
        fh.copy_(fd, non_blocking=True)
    e1.record(stream)
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    e2e = {"value": replicas_throughput(dof, e2e_ms, world), "unit": "space-time DOF/s", "h2d_bytes_per_step": 8 * dof,
           "d2h_bytes_per_step": 8 * dof, "ms_per_step": e2e_ms}

    # ---- rooflines: every phase from its algorithmic work; the dominant kernel is the nearfield
    peaks = _peaks(P, stream)
    es = 8 if head == P.PFMM_FP64 else 4
    rl = phase_rooflines(phases, info, es, nt, ET, M_X, M_T, peaks, arith="df64" if head == P.PFMM_FP64 else "fp32")
    nf = rl["nearfield"]
    tc = head == P.PFMM_MIXED and bool(info["nf_tensor_cores"] & 1)
    crt = head == P.PFMM_FP64 and bool(info["nf_tensor_cores"] & 1)
    # the tensor-core nearfield kernels are timed alone (CUDA events around their launch on the
    # apply's stream); the nearfield phase adds the input split and the output combination
    kms = phases.get("nf_kernel") or nf["ms"]
    ktiming = ("CUDA events around the kernel's launch" if phases.get("nf_kernel")
               else "the nearfield phase (kernel events unavailable)")
    if crt:
        # FP64 nearfield as exact residue products on the tensor cores: 16 FP16 products per
        # product of the method; per launch the kernel reads 16 FP16 residues (32 bytes) per stored
        # element and per input value, and writes 16 one-byte output residues per output value
        nel = info["nearfield_v_elements"]
        byts = 32.0 * nel + 48.0 * dof
        gbs = byts / (kms * 1e-3) / 1e9
        executed = 16.0 * nf["flops"] / (kms * 1e-3) / 1e12
        roofline = {"bound": "hbm", "kernel": "k_nf_apply_crt", "achieved": gbs, "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
                    "traffic": NF_CRT_DRAM_BYTES_PER_ELEMENT * nel, "traffic_source": NF_CRT_TRAFFIC_SOURCE,
                    "peak_source": "measured copy rate (of measured)", "bytes_per_launch": byts,
                    "ms_per_launch": kms, "timing": ktiming, "nearfield_phase_ms": nf["ms"],
                    "tensor": {"executed_fp16_tflops": executed, "frac_of_fp16_peak": executed / peaks["fp16_tflops"]},
                    "method_fp64_tflops": nf["flops"] / (kms * 1e-3) / 1e12, "fp64_pipe_tflops": peaks["fp64_tflops"]}
    elif tc:
        gbs = nf["bytes"] / (kms * 1e-3) / 1e9
        tfl = nf["flops"] / (kms * 1e-3) / 1e12
        roofline = {"bound": "hbm", "kernel": "k_nf_apply_tc", "achieved": gbs, "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"], "traffic": None,
                    "peak_source": "measured copy rate (of measured)", "bytes_per_launch": nf["bytes"],
                    "ms_per_launch": kms, "timing": ktiming, "nearfield_phase_ms": nf["ms"],
                    "tensor": {"algorithmic_tflops": tfl, "frac_of_fp16_peak": tfl / peaks["fp16_tflops"]}}
    else:
        roofline = {"bound": "alu", "kernel": "k_nf_apply<double>" if es == 8 else "k_nf_apply<float>",
                    "achieved": nf["tflops"], "peak": peaks["fp64_tflops"] if es == 8 else peaks["fp32_tflops"],
                    "unit": "TFLOP/s", "frac": nf["frac_fp"], "traffic": None,
                    "peak_source": "FMA rate measured in this run by pfmm_probe_fma_rate (independent FMA chains)",
                    "flops_per_launch": nf["flops"], "ms_per_launch": nf["ms"],
                    "hbm": {"achieved_gbs": nf["gbs"], "frac": nf["frac_hbm"], "bytes_per_launch": nf["bytes"]}}

    # ---- the other precision of the same workload, and the errors between them
    other_line = None
    fo = torch.empty_like(f)
    P.pfmm_apply_V(op.h, w, f, 1, stream)
    torch.cuda.synchronize()
    if args.other_steps > 0:
        op2, t_build2 = build(other)
        ms2, ph2 = run_device_timed(args.other_steps, 1, op2, fo)
        P.pfmm_apply_V(op2.h, w, fo, 1, stream)
        torch.cuda.synchronize()
        f64, fmx = (f, fo) if head == P.PFMM_FP64 else (fo, f)
        rel = float((fmx - f64).abs().max() / f64.abs().max())
        info2 = op2.info()
        other_line = {"precision": "mixed" if other == P.PFMM_MIXED else "fp64",
                      "value": dof / (statistics.mean(ms2) * 1e-3), "ms_per_step": statistics.mean(ms2),
                      "phases_ms": ph2, "build_s": t_build2, "mixed_vs_fp64_rel_maxnorm": rel,
                      "rooflines": phase_rooflines(ph2, info2, 8 if other == P.PFMM_FP64 else 4, nt, ET, M_X, M_T,
                                                   peaks, arith="df64" if other == P.PFMM_FP64 else "fp32"),
                      "nf_tensor_cores": info2["nf_tensor_cores"]}
        op2.close()

    # ---- oracle: cpu_baseline (a matvec on every 64th target row) and parity on those rows
    cpu, parity = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            wn = w[0].cpu().numpy()
            outs = {("fp64" if head == P.PFMM_FP64 else "mixed"): f[0].cpu().numpy()}
            if other_line:
                outs[other_line["precision"]] = fo[0].cpu().numpy()
            cpu, rows, fref = _cpu_baseline(V, T, ET, wn)
            den = np.max(np.abs(fref))
            parity = {"rows": int(len(rows)), "vs_oracle_pfmm": {k: float(np.max(np.abs(v[:, rows] - fref)) / den)
                                                                  for k, v in outs.items()}}
            if args.dense_rows > 0:
                parity["vs_dense_oracle"], parity["dense_rows"] = _dense_rows_error(V, T, ET, wn, outs, args.dense_rows)
        except Exception as e:  # the baseline is context; the line still prints
            cpu = {"value": None, "error": str(e)}

    solve = None
    if rank == 0 and not args.no_solve:
        solve = _solve_comparison(dev, n_test=args.solve_sets)
    batch = None
    if rank == 0 and args.batch > 0:
        batch = _batch_comparison(dev, args.batch)

    if rank == 0:
        cfg = _config_dict(nt, world)
        cfg.update({"precision": args.precision, "build_s": t_build,
                    "nearfield_GB": info["nearfield_bytes"] / 1e9, "nf_form": info["nf_form"],
                    "nf_form_ms_at_build": info["nf_form_ms"], "m2l_engine": info["m2l_engine"],
                    "arithmetic": ("FP64-accurate: nearfield as exact integer products of residues modulo 16 primes "
                                   "(FP16 tcgen05 MMAs, exact FP32 accumulation, Garner's combination to FP64); FMM "
                                   "passes in double-FP32 (two FP32 words, about 48 significant bits); FP64 in / out"
                                   if head == P.PFMM_FP64 else
                                   "mixed: nearfield as three FP16 products of scaled hi / lo parts on tcgen05 with "
                                   "FP32 accumulation; FMM passes in FP32; FP64 in / out")})
        line = {"metric": METRIC, "value": value, "unit": "space-time DOF/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if head == P.PFMM_FP64 else "f32", "data": "synthetic",
                "config": cfg, "phases_ms": phases, "roofline": roofline, "phase_rooflines": rl, "peaks": peaks,
                "cpu_baseline": cpu, "parity": parity, "e2e": e2e, "gpu_launches": launches * args.steps,
                "launches_per_apply": launches, "clocks": _clocks_summary(samples),
                ("mixed" if other == P.PFMM_MIXED else "fp64"): other_line, "solve": solve, "batch": batch}
        print(json.dumps(line), flush=True)
    op.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

"""Benchmark: pFMM V_h matvec throughput (space-time DOF/s) on one GB300.

Workload (the single large problem): surface of the unit cube, 32 x 32 squares per face cut
into 12288 flat triangles, 256 uniform steps on [0, 1] (3,145,728 space-time DOFs), Chebyshev
degree 6 in space, Lagrange degree 4 in time, c_st = 1, temporal leaves of 2 steps.  A step is
one f = V_h w (the product every GMRES iteration applies), w ~ N(0,1) seeded.  The nearfield
blocks and tables are built before the timed region (assembly).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64] [--impl ours|reference]

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
N_A, ET, M_X, M_T, C_ST = 32, 256, 6, 4, 1.0
# DRAM bytes (read + write) per stored panel element of one tensor-core nearfield launch, from an
# ncu capture of the 3072-triangle x 128-step case (None: not captured for the current kernel)
NF_TC_DRAM_BYTES_PER_ELEMENT = 4.79


def _set_size(n_a, et):
    global N_A, ET
    N_A, ET = n_a, et


def _clock_sampler(stop, out):
    cmd = ["nvidia-smi", "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
           "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
           "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-i",
           os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or "0"]
    while not stop.is_set():
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=5)
            if r.returncode == 0:
                out.append(r.stdout.strip().splitlines()[0])
        except Exception:
            pass
        stop.wait(0.2)


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


def _oracle_sample(n_targets=16, nthreads=0):
    """Time the CPU oracle (plain FP64 pFMM of Alg. 2) on a bounded sample: the rows of
    ``n_targets`` triangles (all 256 steps) of the same workload."""
    import oracle as O
    from paper_2106_15911_gb300.inputs import cube_mesh, random_density, sample_triangles

    V, T = cube_mesh(N_A)
    P = O.make_problem(V, T, 1.0, ET, m_t=M_T, m_x=M_X, c_st=C_ST)
    w = random_density(ET, T.shape[0], 1, seed=1234)[0]
    tg = sample_triangles(T.shape[0], n_targets, seed=7)
    t0 = time.perf_counter()
    O.pfmm_apply(P, 0, w, targets=tg, nthreads=nthreads)
    dt = time.perf_counter() - t0
    cores = nthreads if nthreads > 0 else (os.cpu_count() or 1)
    return dict(value=n_targets * ET / dt, unit="space-time DOF/s", cores=cores, kind="oracle",
                sample=f"rows of {n_targets} seeded target triangles x {ET} steps of V_h w (full S2M/M2M, "
                       f"M2L/L2L/L2T on their box chains, their nearfield rows); {dt:.1f} s"), dt


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
    B.close()
    best = min(graph_ms.values())
    mx = [int(p[5].m_x) for p in probs]
    return {"workload": f"{n_problems} problems, 768..12288 triangles, 32..256 steps, 1..8 rhs, mixed, "
                        f"autotuned m_x (truncation estimate {tol:g})",
            "space_time_dofs": dofs, "graph_ms_by_streams": graph_ms, "sequential_ms": t_seq,
            "dofs_per_s": dofs / (best * 1e-3), "build_s": t_build,
            "m_x_histogram": {str(m): mx.count(m) for m in sorted(set(mx))}}


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


def _profile_case(dev, case):
    """Small cases for ncu captures of kernels the matvec does not launch: the learned
    preconditioner's layers (`mpnn`), its compiled form (`mpnn_compiled`), the on-the-fly
    nearfield (`otf`), the slab M2L of 8^3 grids (`m2l_slab`).  3072-triangle cube; 128 steps
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
    return {"profile_case": case, "ms_per_call": e0.elapsed_time(e1) / 2}


def _launches_per_apply(info, nrhs, na=M_T + 1, split_ctas=8 * 152):
    """Kernels one V_h apply launches: permute in and out, the FP16 input split (max |x| and
    split; tensor-core nearfield), nearfield, S2M (per-tile moments and their temporal sum),
    M2M (levels p-1..2), M2L (levels 2..p) plus one term sum per split level (levels with fewer
    than eight (interval, node) CTAs per SM), L2L (levels 3..p), L2T (temporal factor and
    per-tile evaluation).  The two-stage S2M / L2T forms are the ones taken when the M2L
    workspace holds their intermediates, as it does for the bench workload."""
    p = info["p"]
    tc = 2 if info["nf_tensor_cores"] & 1 else 0
    if p < 2:
        return 3 + tc
    split = sum(1 for l in range(2, p + 1) if (2 ** l) * na * nrhs < split_ctas)
    return 2 + tc + 1 + 2 + (p - 2) + (p - 1) + split + (p - 2) + 2


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
    if rank != 0:
        return 0
    vals, tot = [], 0.0
    for _ in range(args.warmup):
        _oracle_sample()
    for _ in range(args.steps):
        cb, dt = _oracle_sample()
        vals.append(cb["value"])
        tot += dt
    v = statistics.mean(vals)
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "space-time DOF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": f"cube {N_A}x{N_A} faces ({12 * N_A * N_A} tri) x {ET} steps",
                                             "m_x": M_X, "m_t": M_T, "c_st": C_ST},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "space-time DOF/s", "h2d_bytes_per_step": 0,
                                          "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true", help="skip the solver comparison")
    ap.add_argument("--solve-sets", type=int, default=32, help="held-out data sets of the solver comparison")
    ap.add_argument("--config5", action="store_true", help="run only the 50M-DOF combined workload")
    ap.add_argument("--config5-matvec", action="store_true",
                    help="with --config5: the build and matvecs only (no recording, training or solves)")
    ap.add_argument("--profile-case", choices=["mpnn", "mpnn_compiled", "otf", "m2l_slab"], default=None,
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
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    V, T = cube_mesh(N_A)
    nt, nv = T.shape[0], V.shape[0]
    dof = nt * ET
    stream = torch.cuda.current_stream()
    prec = P.PFMM_MIXED if args.precision == "mixed" else P.PFMM_FP64

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    t_build = time.perf_counter()
    op = P.Operator(V, T, 1.0, ET, m_t=M_T, m_x=M_X, c_st=C_ST, precision=prec)
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t_build
    info = op.info()
    w = torch.tensor(random_density(ET, nt, 1, seed=1234 + rank), device=dev)
    f = torch.empty_like(w)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2

    def run_device_timed(steps, warm, opx, prof):
        P.pfmm_set_profiling(opx.h, False)
        for _ in range(warm):
            P.pfmm_apply_V(opx.h, w, f, 1, stream)
        P.pfmm_phase_times(opx.h)
        P.pfmm_set_profiling(opx.h, prof)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        barrier()
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(stream)
            P.pfmm_apply_V(opx.h, w, f, 1, stream)
            ev[i][1].record(stream)
        barrier()
        ms = [a.elapsed_time(b) for a, b in ev]
        phases, n = P.pfmm_phase_times(opx.h)
        P.pfmm_set_profiling(opx.h, False)
        return ms, {k: v / max(n, 1) for k, v in phases.items()}

    # ---- timed region (device), with live clock sampling
    stop, samples = threading.Event(), []
    th = threading.Thread(target=_clock_sampler, args=(stop, samples), daemon=True)
    th.start()
    ms, phases = run_device_timed(args.steps, args.warmup, op, prof=True)
    stop.set()
    th.join(timeout=5)
    ms_step = max_over_ranks(statistics.mean(ms), world, dev)
    value = replicas_throughput(dof, ms_step, world)

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

    # ---- roofline of the dominant kernel (nearfield apply): algorithmic work per launch
    ls = 2
    nint = ET // ls
    flops_nf = 2.0 * nt * nt * nint * sum(ls + s + 1 for s in range(ls))  # 2 * E_x^2 * sum_t |D(t)|
    nf_ms = phases["nearfield"]
    fp64 = prec == P.PFMM_FP64
    tc = bool(info.get("nf_tensor_cores", 0) & 1)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    if tc:
        # tcgen05 kind::f16 with a 3-term split: three FP16 products per useful product; the FP16
        # dense rate is the BF16 rate, so the peak is the measured dense BF16 burst peak
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
        bf16 = float(peaks.get("bf16_tflops", 1900.0))
        peak_f16 = bf16
        achieved = 3.0 * flops_nf / (nf_ms * 1e-3) / 1e12
        # algorithmic HBM bytes: the hi/lo FP16 parts of every stored panel element, read once
        bytes_nf = 4.0 * info["nearfield_v_elements"]
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        # DRAM bytes per panel element of this kernel, measured with ncu on the 3072-triangle x
        # 128-step case
        traffic = NF_TC_DRAM_BYTES_PER_ELEMENT * info["nearfield_v_elements"] if NF_TC_DRAM_BYTES_PER_ELEMENT else None
        roofline = {"bound": "tensor", "kernel": "k_nf_apply_tc", "achieved": achieved, "peak": peak_f16,
                    "unit": "TFLOP/s", "frac": achieved / peak_f16, "traffic": traffic,
                    "peak_source": f"measured dense bf16 burst {bf16:.0f} TF = the fp16 rate (of measured)",
                    "flops_per_launch_executed": 3.0 * flops_nf, "ms_per_launch": nf_ms,
                    "hbm": {"achieved_gbs": bytes_nf / (nf_ms * 1e-3) / 1e9, "peak_gbs": hbm,
                            "frac": bytes_nf / (nf_ms * 1e-3) / 1e9 / hbm, "bytes_per_launch": bytes_nf}}
    else:
        peak_meas = P.pfmm_probe_fma_rate(fp64, stream)
        peak_nominal = sm_count * 128 * 2 * 2.07e9 / 1e12  # FP32 lanes x 2 flops x max SM clock
        roofline = {"bound": "alu", "kernel": "k_nf_apply", "achieved": flops_nf / (nf_ms * 1e-3) / 1e12,
                    "peak": peak_meas, "unit": "TFLOP/s", "frac": flops_nf / (nf_ms * 1e-3) / 1e12 / peak_meas,
                    "traffic": None, "peak_source": f"measured {'FP64' if fp64 else 'FP32'} FMA probe "
                                                    f"(nominal FP32 {peak_nominal:.1f} at 2070 MHz)",
                    "flops_per_launch": flops_nf, "ms_per_launch": nf_ms}

    # ---- FP64 mode of the same workload (context; the other half of the workload's comparison)
    fp64_line = None
    if not fp64 and args.fp64_steps > 0:
        op64 = P.Operator(V, T, 1.0, ET, m_t=M_T, m_x=M_X, c_st=C_ST, precision=P.PFMM_FP64)
        ms64, ph64 = run_device_timed(args.fp64_steps, 1, op64, prof=True)
        with torch.no_grad():
            P.pfmm_apply_V(op64.h, w, fd, 1, stream)
            P.pfmm_apply_V(op.h, w, f, 1, stream)
            torch.cuda.synchronize()
            rel = float((f - fd).abs().max() / fd.abs().max())
        fp64_line = {"value": dof / (statistics.mean(ms64) * 1e-3), "ms_per_step": statistics.mean(ms64),
                     "phases_ms": ph64, "mixed_vs_fp64_rel_maxnorm": rel,
                     "fp64_fma_tflops": P.pfmm_probe_fma_rate(True, stream)}
        op64.close()

    solve = None
    if rank == 0 and not args.no_solve:
        solve = _solve_comparison(dev, n_test=args.solve_sets)
    batch = None
    if rank == 0 and args.batch > 0:
        batch = _batch_comparison(dev, args.batch)

    launches = _launches_per_apply(info, 1)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu, _ = _oracle_sample()
        except Exception as e:  # the baseline is context; the line still prints
            cpu = {"value": None, "error": str(e)}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "space-time DOF/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if not fp64 else "f64", "data": "synthetic",
                "config": {"workload": f"cube {N_A}x{N_A} faces ({nt} tri) x {ET} steps, V_h matvec",
                           "dofs": dof, "m_x": M_X, "m_t": M_T, "c_st": C_ST, "precision": args.precision,
                           "l2": "flushed (256 MB write) between timed steps; nearfield blocks "
                                 f"{info['nearfield_bytes'] / 1e9:.2f} GB > L2",
                           "parallelism": f"replicas x{world}", "build_s": t_build},
                "phases_ms": phases, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches * args.steps, "clocks": _clocks_summary(samples), "fp64": fp64_line,
                "solve": solve, "batch": batch}
        print(json.dumps(line), flush=True)
    op.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

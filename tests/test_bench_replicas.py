"""The multi-GPU form of the bench is "replicas only" (no collective in the data path): the
job's throughput is all ranks' units over the slowest rank's time.  The host-side reduction is
run here with world size 2 on the gloo backend (CPU), as bench.py runs it with NCCL."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [3.0, 5.0][rank]  # rank 1 is the slower replica
    m = bench.max_over_ranks(ms, world, "cpu")
    out[rank] = (m, bench.replicas_throughput(1000.0, m, world))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_max_time_and_aggregate_throughput():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
        res = dict(out)
    for r in (0, 1):
        m, v = res[r]
        assert m == 5.0  # every rank sees the slowest time
        assert v == pytest.approx(2 * 1000.0 / 5e-3)


def test_single_rank_needs_no_collective():
    assert bench.max_over_ranks(4.0, 1, None) == 4.0
    assert bench.replicas_throughput(10.0, 2.0, 1) == pytest.approx(5000.0)


def test_phase_rooflines_follow_the_algorithmic_work():
    """Per-phase rooflines of the bench line: the nearfield of the 12288-triangle x 256-step
    workload does 2 x 12288^2 x 128 x 7 flops (the d = 0..2 / 0..3 offsets of the two steps of
    each leaf interval) on 4 x 12288^2 stored FP64 entries; M2L takes the library's count of the
    separable passes; fractions divide by the given peaks."""
    info = {"p": 7, "nbox": [1, 1, 1, 1, 8, 8, 56, 56], "n_m2l_pairs": 1000, "m2l_flops": 3e9,
            "nearfield_v_elements": 4 * 12288 * 12288, "nf_tensor_cores": 0}
    peaks = {"hbm_gbs": 1000.0, "fp64_tflops": 1.0, "fp32_tflops": 50.0}
    rl = bench.phase_rooflines({"nearfield": 100.0, "m2l": 2.0, "s2m": 1.0, "l2t": 1.0}, info, 8, 12288, 256, 6, 4,
                               peaks)
    nf = rl["nearfield"]
    assert nf["flops"] == 2.0 * 12288 ** 2 * 128 * 7
    assert nf["bytes"] == 8.0 * 4 * 12288 ** 2 + 16.0 * 12288 * 256
    assert nf["tflops"] == pytest.approx(nf["flops"] / 0.1 / 1e12)
    assert nf["frac_fp"] == pytest.approx(nf["tflops"] / 1.0) and nf["bound"] == "fp"
    assert rl["m2l"]["flops"] == 3e9
    assert rl["s2m"]["frac_hbm"] == pytest.approx(rl["s2m"]["gbs"] / 1000.0)
    # mixed precision with the tensor-core nearfield: 4 bytes per element; every product of the
    # method is three FP16 products (hi / lo parts), so its attainable rate is the FP16 peak / 3
    info["nf_tensor_cores"] = 3
    rl = bench.phase_rooflines({"nearfield": 1.0}, info, 4, 12288, 256, 6, 4, dict(peaks, fp16_tflops=2000.0))
    assert rl["nearfield"]["bytes"] == 4.0 * 4 * 12288 ** 2 + 16.0 * 12288 * 256
    assert rl["nearfield"]["frac_fp"] == pytest.approx(rl["nearfield"]["tflops"] / (2000.0 / 3))

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


def test_launches_per_apply_matches_the_launch_list():
    """The bench's `gpu_launches` claim counts the kernels of one V_h apply from the tree depth:
    the 12288-triangle x 256-step workload (7 levels, tensor-core nearfield, every M2L level
    split) launches 31, as the ncu launch list of that workload shows; without the tensor-core
    engine the input max and split are not launched; a tree without far field launches the
    permutes and the nearfield only."""
    assert bench._launches_per_apply({"p": 7, "nf_tensor_cores": 3}, 1) == 31
    assert bench._launches_per_apply({"p": 7, "nf_tensor_cores": 0}, 1) == 29
    # more right-hand sides fill the coarse levels: levels with >= 8 CTAs per SM are not split
    assert bench._launches_per_apply({"p": 7, "nf_tensor_cores": 3}, 2) == 30
    assert bench._launches_per_apply({"p": 1, "nf_tensor_cores": 0}, 1) == 3

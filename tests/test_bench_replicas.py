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

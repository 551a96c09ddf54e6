"""Temporal decomposition of the FMM over several ranks (Section 4), emulated on CPU ranks.

The owners of the temporal clusters follow the paper's three rules; its example (16 time slices,
8 processes: level-1 clusters on ranks 1 and 5, level-2 clusters on the owners of their left
children, M2L work W_6 = 3 M2L(4) + 1 M2L(3) + 2 M2L(2) and W_7 = 3 M2L(4) + 2 M2L(3)) is
pinned.  The message plan is then executed by 2, 3, 4 and 8 gloo ranks on CPU on a stand-in of
the FMM with the same data flow on the temporal tree (integer-valued S2M, M2M, M2L over Eq.
03:ILtemp, L2L, L2T and the two-interval nearfield): every rank computes only the clusters it
owns, from its own data and the messages it received, and its part of the result equals the
sequential evaluation exactly.  A rank that needed a value it neither owns nor received would
fail with a KeyError."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from paper_2106_15911_gb300 import pfmm as P  # noqa: E402


def _ilist(k):
    """Temporal interaction list of interval k (Eq. 03:ILtemp)."""
    if k < 2:
        return []
    return [k - 2] if k % 2 == 0 else [k - 3, k - 2]


def test_owners_follow_the_papers_example():
    own = P.pfmm_shard_owners(4, 8)
    assert own[4] == [r for r in range(8) for _ in range(2)] and own[3] == list(range(8))
    assert own[2] == [0, 2, 4, 6]   # the owner of the left child
    assert own[1] == [1, 5]         # the fewest clusters in groups 0-3 and 4-7
    # M2L operations (target clusters times their interaction lists) of ranks 6 and 7, per level
    work = {r: [sum(len(_ilist(k)) for k, o in enumerate(own[l]) if o == r) for l in range(5)] for r in (6, 7)}
    assert work[6][2:] == [2, 1, 3] and work[7][2:] == [0, 2, 3]


@pytest.mark.parametrize("levels,nranks", [(3, 1), (4, 8), (5, 3), (6, 5)])
def test_every_rank_owns_and_messages_are_one_per_destination(levels, nranks):
    own = P.pfmm_shard_owners(levels, nranks)
    assert all(0 <= o < nranks for lev in own for o in lev)
    assert sorted(set(own[levels])) == list(range(min(nranks, 1 << levels)))
    m = P.pfmm_shard_messages(levels, nranks)
    keys = {tuple(r[[0, 1, 2, 4]]) for r in m}
    assert len(keys) == len(m) and all(r[3] != r[4] for r in m)
    if nranks == 1:
        assert len(m) == 0


# ---- the stand-in computation -----------------------------------------------------------------
def _m2l_coef(l, d):
    return 10 * (l + 1) + d


def _sequential(x, levels):
    n = 1 << levels
    M = {(levels, k): int(x[k]) for k in range(n)}
    for l in range(levels - 1, 1, -1):
        for k in range(1 << l):
            M[(l, k)] = M[(l + 1, 2 * k)] + 2 * M[(l + 1, 2 * k + 1)]
    L = {}
    for l in range(2, levels + 1):
        for k in range(1 << l):
            v = sum(_m2l_coef(l, k - J) * M[(l, J)] for J in _ilist(k))
            if l >= 3:
                v += (3 if k % 2 == 0 else 5) * L[(l - 1, k // 2)]
            L[(l, k)] = v
    return [L.get((levels, k), 0) + 7 * int(x[k]) + (11 * int(x[k - 1]) if k else 0) for k in range(n)]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _exchange(rank, msgs, kind, level, have):
    """Send this rank's values of (kind, level) to their destinations, receive the ones addressed
    to it (tag = the cluster), in the plan's order."""
    reqs = []
    for k_, l_, c, src, dst in msgs:
        if k_ == kind and l_ == level and src == rank:
            reqs.append(dist.isend(torch.tensor([have[(l_, c)]], dtype=torch.int64), dst, tag=c))
    got = {}
    for k_, l_, c, src, dst in msgs:
        if k_ == kind and l_ == level and dst == rank:
            t = torch.zeros(1, dtype=torch.int64)
            dist.recv(t, src, tag=c)
            got[(l_, c)] = int(t.item())
    for r in reqs:
        r.wait()
    return got


def _rank(rank, world, port, levels, x, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    own = P.pfmm_shard_owners(levels, world)
    msgs = [tuple(int(v) for v in r) for r in P.pfmm_shard_messages(levels, world)]
    mine = lambda l: [k for k, o in enumerate(own[l]) if o == rank]  # noqa: E731
    n = 1 << levels
    # M-list, bottom up: S2M at the leaves, M2M above; moments to parents and M2L targets
    M = {}
    for l in range(levels, 1, -1):
        for k in mine(l):
            M[(l, k)] = int(x[k]) if l == levels else M[(l + 1, 2 * k)] + 2 * M[(l + 1, 2 * k + 1)]
        M.update(_exchange(rank, msgs, P.PFMM_MSG_MOMENTS, l, M))
    # M2L- and L-lists, top down: locals of a level are final before they go to the children
    L = {}
    for l in range(2, levels + 1):
        for k in mine(l):
            v = sum(_m2l_coef(l, k - J) * M[(l, J)] for J in _ilist(k))
            if l >= 3:
                v += (3 if k % 2 == 0 else 5) * L[(l - 1, k // 2)]
            L[(l, k)] = v
        if l < levels:
            L.update(_exchange(rank, msgs, P.PFMM_MSG_LOCALS, l, L))
    # N-list: the input of the previous leaf interval (halo), then L2T + nearfield
    X = {(levels, k): int(x[k]) for k in mine(levels)}
    X.update(_exchange(rank, msgs, P.PFMM_MSG_INPUT, levels, X))
    f = {k: L.get((levels, k), 0) + 7 * X[(levels, k)] + (11 * X[(levels, k - 1)] if k else 0) for k in mine(levels)}
    out[rank] = f
    dist.barrier()
    dist.destroy_process_group()
    assert n == len(own[levels])


@pytest.mark.parametrize("levels,world", [(4, 2), (5, 3), (4, 4), (4, 8)])
def test_distributed_product_on_cpu_ranks_matches_sequential(levels, world):
    x = np.random.default_rng(levels * 10 + world).integers(-50, 50, 1 << levels)
    ref = _sequential(x, levels)
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, _free_port(), levels, x, out), nprocs=world, start_method="spawn",
                           join=True)
        res = dict(out)
    got = {}
    for r in range(world):
        for k, v in res[r].items():
            assert k not in got
            got[k] = v
    assert [got[k] for k in range(1 << levels)] == ref

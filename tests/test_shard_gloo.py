"""Sharding of independent products across ranks, run as world-size-2 gloo
process groups on the CPU: every rank derives the same assignment, each graph
(and each right-hand-side column) is owned by exactly one rank, and the
timing reduction gives the max time and the total units on every rank."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1708_07271_gb300 import shard


def test_assign_graphs_covers_and_balances():
    sizes = [5, 100, 7, 100, 3, 60, 40, 1, 0]
    for world in (1, 2, 3, 4, 16):
        parts = shard.assign_graphs(sizes, world)
        assert len(parts) == world
        owned = sorted(i for p in parts for i in p)
        assert owned == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in parts]
        # longest-first greedy: max load <= mean + largest item
        assert max(loads) <= sum(sizes) / world + max(sizes)
    assert shard.assign_graphs(sizes, 2) == shard.assign_graphs(list(sizes), 2)  # deterministic


@pytest.mark.parametrize("k", [0, 1, 5, 32, 33])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_column_slices_partition(k, world):
    cols = []
    for r in range(world):
        lo, hi = shard.column_slice(k, world, r)
        assert 0 <= lo <= hi <= k and hi - lo in (k // world, k // world + 1)
        cols += list(range(lo, hi))
    assert cols == list(range(k))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, sizes, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        parts = shard.assign_graphs(sizes, world)
        mine = parts[rank]
        units = sum(sizes[i] for i in mine)
        seconds = 0.25 * (rank + 1)  # a stand-in for each rank's measured time
        t, u = shard.reduce_timing(seconds, units)
        # every rank sees the same partition (gathered and compared)
        gathered = [None] * world
        dist.all_gather_object(gathered, parts)
        q.put((rank, t, u, all(g == parts for g in gathered), mine))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    sizes = [3, 9, 27, 81, 1, 2, 50]
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, sizes, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, t, u, same, mine in res:
        assert t == 0.25 * world  # max over ranks
        assert u == sum(sizes)  # every edge counted once
        assert same
    assert sorted(res[0][4] + res[1][4]) == list(range(len(sizes)))

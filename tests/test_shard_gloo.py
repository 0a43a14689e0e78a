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


# ---------------------------------------------------------------- row shards
import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402


def test_row_blocks_and_masked_csr():
    g = synth.copying_model(synth.tiny_web())
    for world in (1, 2, 3, 4):
        blocks = shard.row_blocks(g.row_ptr, world)
        assert blocks[0][0] == 0 and blocks[-1][1] == g.n
        assert all(blocks[r][1] == blocks[r + 1][0] for r in range(world - 1))
        edges = [g.row_ptr[b] - g.row_ptr[a] for a, b in blocks]
        assert max(edges) - min(edges) <= 2 * np.diff(g.row_ptr).max() + 1
        x = synth.rhs(g.n, 2, 5).astype(np.float64)
        total_xA = np.zeros_like(x)
        for a, b in blocks:
            rp, ci = shard.masked_csr(g.row_ptr, g.col, a, b)
            assert rp[-1] == len(ci) and np.all(np.diff(rp[:a + 1]) == 0) and np.all(np.diff(rp[b:]) == 0)
            total_xA += oracle.csr_xA(rp, ci, x)
            np.testing.assert_allclose(oracle.csr_Ax(rp, ci, x)[a:b], oracle.csr_Ax(g.row_ptr, g.col, x)[a:b])
        np.testing.assert_allclose(total_xA, oracle.csr_xA(g.row_ptr, g.col, x), rtol=1e-12)


def test_masked_encoding_keeps_references_inside_the_block():
    import paper_1708_07271_gb300 as bvg
    g = synth.copying_model(synth.tiny_web())
    for a, b in shard.row_blocks(g.row_ptr, 3):
        rp, ci = shard.masked_csr(g.row_ptr, g.col, a, b)
        ref, _ = bvg.bvg_get_refs(bvg.bvg_encode(rp, ci))
        inside = ref[a:b]
        assert np.all((inside == -1) | ((inside >= a) & (inside < np.arange(a, b))))
        assert np.all(ref[:a] == -1) and np.all(ref[b:] == -1)


def _row_worker(rank, world, port, q):
    import torch
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = synth.copying_model(synth.replace(synth.tiny_web(), n=3000, seed=21))
        blocks = shard.row_blocks(g.row_ptr, world)
        rp, ci = shard.masked_csr(g.row_ptr, g.col, *blocks[rank])
        # the CPU stand-in for this rank's device products: the oracle on the masked CSR
        local_Ax = lambda x: torch.from_numpy(oracle.csr_Ax(rp, ci, x.numpy().astype(np.float64)).astype(np.float32))  # noqa: E731
        local_xA = lambda x: torch.from_numpy(oracle.csr_xA(rp, ci, x.numpy().astype(np.float64)).astype(np.float32))  # noqa: E731
        sh = shard.RowSharded(g.n, blocks, rank, local_Ax, local_xA)
        x = torch.from_numpy(synth.rhs(g.n, 3, 9))
        ax = sh.Ax(x).numpy()
        xa = sh.xA(x).numpy()
        xa_owned = sh.xA_owned(x).numpy()
        deg = np.diff(g.row_ptr)
        inv = torch.from_numpy(np.where(deg > 0, 1.0 / np.maximum(deg, 1), 0).astype(np.float32))
        p, it, res = sh.pagerank(inv, tol=1e-9)
        q.put((rank, ax, xa, p.numpy(), it, res, xa_owned, blocks[rank]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3, 4])
def test_row_sharded_products_and_pagerank(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_row_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=180) for _ in range(world)], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = synth.copying_model(synth.replace(synth.tiny_web(), n=3000, seed=21))
    x = synth.rhs(g.n, 3, 9).astype(np.float64)
    want_ax, want_xa = oracle.csr_Ax(g.row_ptr, g.col, x), oracle.csr_xA(g.row_ptr, g.col, x)
    pstar, _, _ = oracle.pagerank(g.row_ptr, g.col, alpha=0.15, tol=1e-13, max_iter=3000, dangling=1)
    for rank, ax, xa, p, it, r, xa_owned, (lo, hi) in res:
        np.testing.assert_allclose(ax, want_ax, rtol=1e-5, atol=1e-5)
        np.testing.assert_allclose(xa, want_xa, rtol=1e-5, atol=1e-5)
        # the reduce-scatter: this rank's block only, the same sums as the all-reduce
        assert xa_owned.shape == (hi - lo, 3)
        np.testing.assert_allclose(xa_owned, want_xa[lo:hi], rtol=1e-5, atol=1e-5)
        assert r < 1e-9 and np.abs(p - pstar[:, 0]).sum() <= 1e-6
    assert [b for *_, b in res] == shard.row_blocks(g.row_ptr, world)
    for other in res[1:]:
        np.testing.assert_array_equal(res[0][3], other[3])  # every rank holds the same iterate

"""Host-side sharding of independent work across ranks (one process per GPU).

The products of different graphs, and of different right-hand-side columns,
share nothing, so ranks split them with no data-path collective; the only
collectives are the timing reductions (max of the elapsed time, sum of the
units processed) that turn per-rank runs into one whole-job figure.
"""
from __future__ import annotations


def assign_graphs(edge_counts, world: int) -> list[list[int]]:
    """Greedy longest-first assignment of graphs to ranks by edge count.

    Every rank computes the same assignment from the same list (ties go to
    the lower rank, graphs of equal size keep their input order). Returns,
    per rank, the ascending list of graph indices it owns."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(edge_counts)), key=lambda i: (-int(edge_counts[i]), i))
    load = [0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += int(edge_counts[i])
    return [sorted(v) for v in out]


def column_slice(k: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous share [lo, hi) of k right-hand-side columns for `rank`
    (sizes differ by at most one; ranks beyond k get an empty slice)."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    base, extra = divmod(k, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def reduce_timing(seconds: float, units: float, group=None, device=None) -> tuple[float, float]:
    """(max of seconds, sum of units) over the ranks of `group` (identity
    without torch.distributed). `device` is where the reduction tensor lives
    (the rank's GPU under NCCL, the CPU under gloo)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(seconds), float(units)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), float(u.item())

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


# ------------------------------------------------------------- row sharding
def row_blocks(row_ptr, world: int) -> list[tuple[int, int]]:
    """Contiguous row blocks [lo, hi), one per rank, with about equal edges
    (block r ends at the first row where the edge prefix reaches (r+1)/world
    of the total)."""
    import numpy as np
    rp = np.asarray(row_ptr, np.int64)
    n, m = len(rp) - 1, int(rp[-1])
    cuts = [0]
    for r in range(1, world):
        cuts.append(max(cuts[-1], int(np.searchsorted(rp, m * r / world, side="left"))))
    cuts.append(n)
    return [(min(cuts[r], n), min(cuts[r + 1], n)) for r in range(world)]


def masked_csr(row_ptr, col, lo: int, hi: int):
    """The CSR of A with every row outside [lo, hi) emptied (same n and ids).
    Encoded on its own, no row of the block takes a reference outside it: an
    empty row can never be a cheaper reference than the raw row."""
    import numpy as np
    rp = np.asarray(row_ptr, np.int64)
    ci = np.asarray(col, np.int32)
    out = np.zeros_like(rp)
    out[lo + 1:hi + 1] = rp[lo + 1:hi + 1] - rp[lo]
    out[hi + 1:] = out[hi]
    return out, ci[rp[lo]:rp[hi]].copy()


class RowSharded:
    """A partitioned by rows over the ranks of the default process group.

    `local_Ax(x)` and `local_xA(x)` compute this rank's products with its
    masked A (full-length vectors, row-major n x k torch tensors on the
    rank's device): the CUDA path on a GPU rank (bvg_spmv_Ax / bvg_spmv_xA on
    the encoding of masked_csr), any stand-in elsewhere. The exchanges:
      A x^T:      each rank forms its own rows; one all-gather of the row
                  blocks;
      x A owned:  each rank forms a full-length partial sum over its rows;
                  one reduce-scatter leaves each rank the sum over all ranks
                  of its own block of entries (a ring moves (P-1)/P of the
                  n x k partial per rank);
      x A:        the same partials, one all-reduce (sum): every rank holds
                  all of y, twice the bytes of the reduce-scatter; the power
                  iteration needs the whole iterate on every rank.
    """

    def __init__(self, n: int, blocks, rank: int, local_Ax, local_xA):
        self.n, self.blocks, self.rank = n, list(blocks), rank
        self.local_Ax, self.local_xA = local_Ax, local_xA

    def Ax(self, x):
        import torch
        import torch.distributed as dist
        lo, hi = self.blocks[self.rank]
        y = self.local_Ax(x)
        width = max(b - a for a, b in self.blocks)
        shape = (width,) + tuple(x.shape[1:])
        mine = torch.zeros(shape, dtype=y.dtype, device=y.device)
        mine[:hi - lo] = y[lo:hi]
        parts = [torch.empty_like(mine) for _ in self.blocks]
        dist.all_gather(parts, mine)
        out = torch.empty_like(y)
        for (a, b), p in zip(self.blocks, parts):
            out[a:b] = p[:b - a]
        return out

    def xA(self, x):
        """All of y = x A on every rank (all-reduce of the partial sums)."""
        import torch.distributed as dist
        y = self.local_xA(x)
        dist.all_reduce(y)
        return y

    def xA_owned(self, x):
        """This rank's block [lo, hi) of y = x A (reduce-scatter of the
        partial sums to the block owners; blocks padded to the widest)."""
        import torch
        import torch.distributed as dist
        y = self.local_xA(x)
        width = max(b - a for a, b in self.blocks)
        rest = tuple(y.shape[1:])
        buf = torch.zeros((len(self.blocks) * width,) + rest, dtype=y.dtype, device=y.device)
        for r, (a, b) in enumerate(self.blocks):
            buf[r * width:r * width + (b - a)] = y[a:b]
        out = torch.empty((width,) + rest, dtype=y.dtype, device=y.device)
        dist.reduce_scatter_tensor(out, buf)
        lo, hi = self.blocks[self.rank]
        return out[:hi - lo]

    def pagerank(self, inv_outdeg, alpha: float = 0.15, tol: float = 1e-8, max_iter: int = 1000):
        """Power iteration of Eq. 1 (uniform teleport, dangling mass returned
        uniformly) on the sharded x A; every rank holds the full iterate.
        Returns (p, iterations, last L1 change)."""
        import torch
        n = self.n
        p = torch.full((n,), 1.0 / n, dtype=torch.float64, device=inv_outdeg.device)
        dang = inv_outdeg == 0
        res = float("inf")
        for it in range(1, max_iter + 1):
            y = self.xA((p * inv_outdeg.to(torch.float64)).to(torch.float32)).to(torch.float64)
            q = alpha / n + (1 - alpha) * (y + p[dang].sum() / n)
            res = float((q - p).abs().sum())
            p = q
            if res < tol:
                return p, it, res
        return p, max_iter, res

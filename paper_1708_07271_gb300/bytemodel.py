"""Algorithmic (compulsory) bytes of each kernel launch, for roofline figures.

Every array a kernel must touch is counted once: structure read once, each
distinct vector element read once, each output written once. Re-reads of
gathered elements (served by L1/L2 when ids are local) are not counted, so
DRAM traffic measured by ncu above these figures means re-reads.

Per launch with k right-hand sides (n rows, layout sizes from bvg_dev_layout):
  push_chain   4n (descendant masks) + 4kn (x) + 4kn (z)
  push_gather  4(n+1) (column offsets) + 4*col_entries + 4(n+1) + 4*tail_items
               (tail items) + 4*(carry_tiles+1) + 4*carry_entries + 4kn (z) + 4kn (y)
  pull         n (meta) + 4(n+1) (item offsets per row) + 4(items+1) (item starts)
               + 4*pull_entries (expanded entries) + 4(n+1) + 8*pull_intervals
               (kept intervals) + 4kn (x) + 4kn (y); the items' partial sums
               (4 bytes per item and right-hand side, written then read back)
               are scratch that stays in L2 at k = 1 and are not counted
  push_gather_pt  (point columns) 4(n+1) (column offsets) + 4*point_entries
               [+ 4(n+1) + 4*point_tail_items (tail items) when k <= 4, where one lane
               group owns a column and the tail items are shared out] + 4kn (z) + 4kn (y)
  csr          8(n+1) (row offsets) + 4m (ids) + 4kn (x) + 4kn (y)
  push_fused   (one right-hand side, one kernel) 4n (descendant masks) + 4(n+1) (column
               offsets) + 2*col_entries (16-bit entries) + 4*(carry_tiles+1) + 4*carry_entries
               + 16*ceil(n/1024) (per-tile row windows) + 4*32*ceil(n/128) (each warp's
               column order) + 1024*ceil(n/1024) (the chain weights' row order) + 4n (x)
               + 4n (y); the chain weights never leave shared
               memory, and the window rows read by two neighbouring tiles come from
               L2 the second time
  pull_fused   (one right-hand side, one kernel; every interval expanded, so the layout's
               pull_items / pull_entries are its items and entries) n (meta) + 4(n+1) (item
               offsets per row) + 4(items+1) (item starts) + 2*pull_entries (16-bit entries)
               + 8*ceil(n/1024) (per-tile column windows) + 4n (x) + 4n (y); the items' and
               rows' sums never leave shared memory
  pr_fused     push_fused + 4n (1/outdeg) [+ 4n (p0) when a teleport vector is
               given]: x is the previous iterate (read once), the new iterate is
               written in place of y
  pr_chain     push_chain + 4n (1/outdeg)
  pr_gather    push_gather - 4kn (y not stored) + 4n (1/outdeg) + 4kn (q_prev)
               + 4kn (q_new) [+ 4kn (p0) when teleport vectors are given]; pr_gather_pt
               likewise from push_gather_pt
"""
from __future__ import annotations


def push_chain(L: dict, k: int) -> int:
    n = L["n"]
    return 4 * n + 8 * k * n


def push_gather(L: dict, k: int) -> int:
    n = L["n"]
    return (4 * (n + 1) + 4 * L["col_entries"] + 4 * (n + 1) + 4 * L.get("tail_items", 0)
            + 4 * (L["carry_tiles"] + 1) + 4 * L["carry_entries"] + 8 * k * n)


def pull(L: dict, k: int) -> int:
    n = L["n"]
    return (n + 4 * (n + 1) + 4 * (L["pull_items"] + 1) + 4 * L["pull_entries"] + 4 * (n + 1)
            + 8 * L["pull_intervals"] + 8 * k * n)


def csr(n: int, m: int, k: int) -> int:
    return 8 * (n + 1) + 4 * m + 8 * k * n


def pr_chain(L: dict, k: int) -> int:
    return push_chain(L, k) + 4 * L["n"]


def pr_gather(L: dict, k: int, with_p0: bool) -> int:
    n = L["n"]
    return push_gather(L, k) - 4 * k * n + 4 * n + 8 * k * n + (4 * k * n if with_p0 else 0)


def push_gather_pt(L: dict, k: int) -> int:
    n = L["n"]
    tail = 4 * (n + 1) + 4 * L["point_tail_items"] if k <= 4 else 0
    return 4 * (n + 1) + 4 * L["point_entries"] + tail + 8 * k * n


def pr_gather_pt(L: dict, k: int, with_p0: bool) -> int:
    n = L["n"]
    return push_gather_pt(L, k) - 4 * k * n + 4 * n + 8 * k * n + (4 * k * n if with_p0 else 0)


def push_fused(L: dict, k: int) -> int:
    n = L["n"]
    return (4 * n + 4 * (n + 1) + 2 * L["col_entries"] + 4 * (L["carry_tiles"] + 1) + 4 * L["carry_entries"]
            + 16 * ((n + 1023) // 1024) + 128 * ((n + 127) // 128) + 1024 * ((n + 1023) // 1024) + 8 * k * n)


def pull_fused(L: dict, k: int) -> int:
    n = L["n"]
    return (n + 4 * (n + 1) + 4 * (L["pull_items"] + 1) + 2 * L["pull_entries"] + 8 * ((n + 1023) // 1024)
            + 8 * k * n)


def pr_fused(L: dict, k: int, with_p0: bool = False) -> int:
    n = L["n"]
    return push_fused(L, k) + 4 * n + (4 * k * n if with_p0 else 0)


def xA_total(L: dict, k: int) -> int:
    return push_chain(L, k) + push_gather(L, k)


KERNELS = {"push_gather": push_gather, "push_gather_pt": push_gather_pt, "push_chain": push_chain, "pull": pull,
           "push_fused": push_fused, "pull_fused": pull_fused}

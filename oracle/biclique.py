"""ORACLE -- test infrastructure only (see the package docstring).

The biclique representation of a binary adjacency matrix, as the paper's
final remarks (Sec. 6) describe it: the edges are split into bicliques
(S_r, C_r), every node of S_r pointing to every node of C_r, plus a set of
residual edges. A biclique's |S_r| * |C_r| edges are stored as the two lists,
|S_r| + |C_r| words.

Products on that representation, in the order the passage gives them:
  A x^T: c_r = sum_{j in C_r} x_j for every biclique; y = 0; for every
         biclique r and every i in S_r, y_i += c_r; then for every residual
         edge A_ij = 1, y_i += x_j.
  x A:   the same with the roles of the two sides swapped (the passage states
         A x^T only; the left product is its transpose): d_r = sum_{i in S_r}
         x_i; y_j += d_r for every j in C_r; then y_j += x_i for every
         residual edge A_ij = 1.
Plain NumPy in FP64, one biclique at a time; no blocking or reordering
beyond the passage's steps.

A decomposition is a dict of CSR-like arrays:
  s_ptr (int64, bicliques + 1), s_idx (int32): the rows S_r
  c_ptr (int64, bicliques + 1), c_idx (int32): the columns C_r
  r_ptr (int64, n + 1), r_col (int32): the residual edges by row
"""
from __future__ import annotations

import numpy as np


def _spans(ptr, idx, r):
    return idx[ptr[r]:ptr[r + 1]].astype(np.int64)


def biclique_Ax(dec: dict, x: np.ndarray) -> np.ndarray:
    """y = A x^T on the biclique representation (Sec. 6); x is n or n x k."""
    x = np.asarray(x, np.float64)
    xs = x.reshape(x.shape[0], -1)
    y = np.zeros_like(xs)
    nb = len(dec["s_ptr"]) - 1
    for r in range(nb):
        c_r = xs[_spans(dec["c_ptr"], dec["c_idx"], r)].sum(axis=0)
        for i in _spans(dec["s_ptr"], dec["s_idx"], r):
            y[i] += c_r
    rp, rc = dec["r_ptr"], dec["r_col"]
    for i in range(len(rp) - 1):
        for j in rc[rp[i]:rp[i + 1]]:
            y[i] += xs[j]
    return y.reshape(x.shape)


def biclique_xA(dec: dict, x: np.ndarray) -> np.ndarray:
    """y = x A on the biclique representation: the transpose of the passage's
    steps (a sum over S_r, added to every column of C_r; residual edges)."""
    x = np.asarray(x, np.float64)
    xs = x.reshape(x.shape[0], -1)
    y = np.zeros_like(xs)
    nb = len(dec["s_ptr"]) - 1
    for r in range(nb):
        d_r = xs[_spans(dec["s_ptr"], dec["s_idx"], r)].sum(axis=0)
        for j in _spans(dec["c_ptr"], dec["c_idx"], r):
            y[j] += d_r
    rp, rc = dec["r_ptr"], dec["r_col"]
    for i in range(len(rp) - 1):
        for j in rc[rp[i]:rp[i + 1]]:
            y[j] += xs[i]
    return y.reshape(x.shape)


def edges_of(dec: dict, n: int) -> np.ndarray:
    """Every edge the representation stores, as sorted (i, j) pairs encoded
    i * n + j, with repeats kept (a valid decomposition has none)."""
    out = []
    nb = len(dec["s_ptr"]) - 1
    for r in range(nb):
        s = _spans(dec["s_ptr"], dec["s_idx"], r)
        c = _spans(dec["c_ptr"], dec["c_idx"], r)
        out.append((s[:, None] * n + c[None, :]).ravel())
    rp = dec["r_ptr"]
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    out.append(rows * n + dec["r_col"].astype(np.int64))
    return np.sort(np.concatenate(out)) if out else np.zeros(0, np.int64)


def words(dec: dict) -> int:
    """Words of the representation: |S_r| + |C_r| per biclique plus one per
    residual edge (Sec. 6)."""
    return int(len(dec["s_idx"]) + len(dec["c_idx"]) + len(dec["r_col"]))

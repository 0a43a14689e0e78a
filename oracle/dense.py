"""ORACLE -- test infrastructure only.

Dense brute force for tiny graphs (n <= a few hundred): the adjacency matrix
as a NumPy array, products by ``@``, and PageRank as the solution of the
linear system its fixed point satisfies (Sec. 3). These pin the C oracle to
something other than itself.
"""
from __future__ import annotations

import numpy as np


def dense_matrix(row_ptr, col, n=None) -> np.ndarray:
    """A_uv = 1 iff v is a successor of u (Sec. 3)."""
    n = len(row_ptr) - 1 if n is None else n
    A = np.zeros((n, n), np.float64)
    for u in range(n):
        for e in range(int(row_ptr[u]), int(row_ptr[u + 1])):
            A[u, int(col[e])] = 1.0
    return A


def pagerank_solve(A: np.ndarray, alpha: float, p0: np.ndarray, dangling: int = 0) -> np.ndarray:
    """Fixed point of p = alpha p0 + (1-alpha) (p D^-1 A + delta(p) p0), with
    delta(p) = sum of p over rows of zero out-degree (spread along g = p0, or
    uniformly with dangling=1), solved directly:
    p [I - (1-alpha)(M + e_dangling g^T)] = alpha p0 (numpy.linalg.solve)."""
    n = A.shape[0]
    d = A.sum(axis=1)
    M = np.zeros_like(A)
    nz = d > 0
    M[nz] = A[nz] / d[nz, None]
    dang = (~nz).astype(np.float64)
    p0 = np.asarray(p0, np.float64).reshape(n)
    g = p0 if dangling == 0 else np.full(n, 1.0 / n)
    T = M + np.outer(dang, g)
    lhs = np.eye(n) - (1.0 - alpha) * T
    # row vector p: p @ lhs = alpha p0  <=>  lhs^T p^T = alpha p0^T
    return np.linalg.solve(lhs.T, alpha * p0)

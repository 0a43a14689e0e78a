"""ORACLE -- test infrastructure only.

Plain, slow, obviously correct FP64 CPU implementation of what the compressed
adjacency products and PageRank compute, written from the paper (Sec. 3-5)
and sharing no code with the CUDA library. Only the test suite,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import it.

C core (oracle.c, compiled with gcc): CSR products by definition, the
reference choice, the sequential compressed product of Sec. 4, the push form
of the left product, nnz(A') counts and PageRank power iteration (Eq. 1).
NumPy parts here: dense brute-force products for tiny graphs (dense.py) and
the warm-start network's forward/backward (mlp.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32


def build(force: bool = False) -> str:
    """Compiles oracle.c into _build/liboracle.so (plain gcc -O2, no fast-math)."""
    src = os.path.join(_HERE, "oracle.c")
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_csr_Ax.argtypes = [_I64, _P, _P, _P, _I32, _P]
            lib.oracle_csr_xA.argtypes = [_I64, _P, _P, _P, _I32, _P]
            lib.oracle_choose_refs.argtypes = [_I64, _P, _P, _I32, _I32, _I32, _P, _P]
            lib.oracle_counts.argtypes = [_I64, _P, _P, _P, _I32, _P]
            lib.oracle_bv_Ax.argtypes = [_I64, _P, _P, _P, _P, _I32, ctypes.c_int, _P]
            lib.oracle_bv_xA.argtypes = [_I64, _P, _P, _P, _P, _I32, ctypes.c_int, _P]
            lib.oracle_chain_weights.argtypes = [_I64, _P, _P, _I32, _P]
            lib.oracle_pagerank.argtypes = [_I64, _P, _P, ctypes.c_double, _P, _P, _I32, ctypes.c_double,
                                            _I32, _I32, _P, _P]
            lib.oracle_pagerank.restype = _I32
            _lib = lib
    return _lib


def _csr(row_ptr, col):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col, dtype=np.int32)
    return rp, ci, len(rp) - 1


def _vec(x, n):
    x = np.ascontiguousarray(x, dtype=np.float64)
    squeeze = x.ndim == 1
    x2 = x.reshape(n, -1)
    return np.ascontiguousarray(x2), x2.shape[1], squeeze


def csr_Ax(row_ptr, col, x):
    """y = A x^T by definition, FP64."""
    rp, ci, n = _csr(row_ptr, col)
    x2, k, sq = _vec(x, n)
    y = np.empty((n, k), np.float64)
    _load().oracle_csr_Ax(n, rp.ctypes.data, ci.ctypes.data, x2.ctypes.data, k, y.ctypes.data)
    return y[:, 0] if sq else y


def csr_xA(row_ptr, col, x):
    """y = x A by definition, FP64."""
    rp, ci, n = _csr(row_ptr, col)
    x2, k, sq = _vec(x, n)
    y = np.empty((n, k), np.float64)
    _load().oracle_csr_xA(n, rp.ctypes.data, ci.ctypes.data, x2.ctypes.data, k, y.ctypes.data)
    return y[:, 0] if sq else y


def choose_refs(row_ptr, col, window=7, max_chain=3, min_interval=4):
    """Reference vector (-1 = none) and chain depths; see oracle.c."""
    rp, ci, n = _csr(row_ptr, col)
    ref = np.empty(n, np.int32)
    depth = np.empty(n, np.int32)
    _load().oracle_choose_refs(n, rp.ctypes.data, ci.ctypes.data, window, max_chain, min_interval,
                               ref.ctypes.data, depth.ctypes.data)
    return ref, depth


COUNT_KEYS = ("dropped", "added", "residual", "intervals", "interval_members", "nnz_diff", "words",
              "rows_with_ref")


def counts(row_ptr, col, ref, min_interval=4) -> dict:
    """nnz(A') and the split of its entries for reference vector ref."""
    rp, ci, n = _csr(row_ptr, col)
    ref = np.ascontiguousarray(ref, dtype=np.int32)
    out = np.zeros(8, np.int64)
    _load().oracle_counts(n, rp.ctypes.data, ci.ctypes.data, ref.ctypes.data, min_interval, out.ctypes.data)
    return dict(zip(COUNT_KEYS, (int(v) for v in out)))


def bv_Ax(row_ptr, col, ref, x, absval=False):
    """y = A x^T by the sequential compressed algorithm of Sec. 4."""
    rp, ci, n = _csr(row_ptr, col)
    ref = np.ascontiguousarray(ref, dtype=np.int32)
    x2, k, sq = _vec(x, n)
    y = np.zeros((n, k), np.float64)
    _load().oracle_bv_Ax(n, rp.ctypes.data, ci.ctypes.data, ref.ctypes.data, x2.ctypes.data, k, int(absval),
                         y.ctypes.data)
    return y[:, 0] if sq else y


def bv_xA(row_ptr, col, ref, x, absval=False):
    """y = x A by pushing x down the reference chains, then applying A'."""
    rp, ci, n = _csr(row_ptr, col)
    ref = np.ascontiguousarray(ref, dtype=np.int32)
    x2, k, sq = _vec(x, n)
    y = np.zeros((n, k), np.float64)
    _load().oracle_bv_xA(n, rp.ctypes.data, ci.ctypes.data, ref.ctypes.data, x2.ctypes.data, k, int(absval),
                         y.ctypes.data)
    return y[:, 0] if sq else y


def chain_weights(ref, x):
    """z_k = sum of x over the rows whose reference chain passes through k."""
    ref = np.ascontiguousarray(ref, dtype=np.int32)
    n = len(ref)
    x2, k, sq = _vec(x, n)
    z = np.empty((n, k), np.float64)
    _load().oracle_chain_weights(n, ref.ctypes.data, x2.ctypes.data, k, z.ctypes.data)
    return z[:, 0] if sq else z


def pagerank(row_ptr, col, alpha=0.15, p0=None, p_init=None, k=None, tol=1e-8, max_iter=1000, dangling=0):
    """PageRank power iteration (Eq. 1) in FP64. p0: n x k teleport vectors
    (default: uniform 1/n, one column). dangling: 0 = mass of zero-out-degree
    rows returns along p0, 1 = uniformly. Returns (p, iterations, residuals)."""
    rp, ci, n = _csr(row_ptr, col)
    if p0 is None:
        p0 = np.full((n, 1 if k is None else k), 1.0 / n)
    p0 = np.ascontiguousarray(np.asarray(p0, np.float64).reshape(n, -1))
    kk = p0.shape[1]
    pi = None if p_init is None else np.ascontiguousarray(np.asarray(p_init, np.float64).reshape(n, kk))
    p = np.empty((n, kk), np.float64)
    resid = np.empty(kk, np.float64)
    it = _load().oracle_pagerank(n, rp.ctypes.data, ci.ctypes.data, float(alpha), p0.ctypes.data,
                                 None if pi is None else pi.ctypes.data, kk, float(tol), int(max_iter),
                                 int(dangling), p.ctypes.data, resid.ctypes.data)
    return p, int(it), resid


from . import dense  # noqa: E402,F401

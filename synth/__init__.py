"""Seeded synthetic inputs shared by the CUDA library's tests/bench and the oracle.

This module holds no arithmetic of the compressed product: it only produces
graphs (CSR of a binary adjacency matrix A) and right-hand-side vectors.
The graphs stand in for the web and social crawls of the paper's Table 1
(Sec. 5), which are not available: a copying model whose rows copy the
successor lists of nearby rows (the copy property of Sec. 4), with local ids
and runs of consecutive ids. See graphgen.c for the model.

Seeds follow seed = 170807271 + 1000 * workload_index + graph_index.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, asdict, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libsynth.so")
_lock = threading.Lock()
_lib = None

BASE_SEED = 170807271


def build(force: bool = False) -> str:
    """Compiles graphgen.c into _build/libsynth.so (gcc, -O2, portable flags)."""
    src = os.path.join(_HERE, "graphgen.c")
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, src])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("seed", ctypes.c_uint64), ("p_copy", ctypes.c_double),
        ("fidelity", ctypes.c_double), ("extra_mean", ctypes.c_double),
        ("fresh_mean", ctypes.c_double), ("powerlaw", ctypes.c_int32), ("alpha", ctypes.c_double),
        ("dmin", ctypes.c_int64), ("dmax", ctypes.c_int64), ("q_run", ctypes.c_double),
        ("run_min", ctypes.c_int32), ("run_max", ctypes.c_int32), ("gap_mean", ctypes.c_double),
        ("random_ids", ctypes.c_int32), ("window", ctypes.c_int32),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.synth_copying_model.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(ctypes.c_void_p),
                                                ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int64)]
            lib.synth_copying_model.restype = ctypes.c_int
            lib.synth_free.argtypes = [ctypes.c_void_p]
            lib.synth_uniform.argtypes = [ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p]
            lib.synth_nodes.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p]
            _lib = lib
    return _lib


@dataclass(frozen=True)
class GraphSpec:
    """Parameters of the copying model (see graphgen.c)."""
    n: int
    seed: int
    p_copy: float = 0.8
    fidelity: float = 0.97
    extra_mean: float = 0.6
    fresh_mean: float = 20.0
    powerlaw: bool = False
    alpha: float = 2.1
    dmin: int = 4
    dmax: int = 20000
    q_run: float = 0.3
    run_min: int = 4
    run_max: int = 20
    gap_mean: float = 40.0
    random_ids: bool = False
    window: int = 7


@dataclass
class Graph:
    """CSR of a binary adjacency matrix: rows sorted, no duplicates."""
    n: int
    row_ptr: np.ndarray  # int64[n+1]
    col: np.ndarray      # int32[m]
    spec: GraphSpec | None = None

    @property
    def m(self) -> int:
        return int(self.row_ptr[-1])


def copying_model(spec: GraphSpec) -> Graph:
    lib = _load()
    p = _Params(spec.n, spec.seed & 0xFFFFFFFFFFFFFFFF, spec.p_copy, spec.fidelity, spec.extra_mean,
                spec.fresh_mean, int(spec.powerlaw), spec.alpha, spec.dmin, spec.dmax, spec.q_run,
                spec.run_min, spec.run_max, spec.gap_mean, int(spec.random_ids), spec.window)
    rp = ctypes.c_void_p()
    ci = ctypes.c_void_p()
    m = ctypes.c_int64()
    rc = lib.synth_copying_model(ctypes.byref(p), ctypes.byref(rp), ctypes.byref(ci), ctypes.byref(m))
    if rc != 0:
        raise ValueError(f"synth_copying_model failed for {spec}")
    try:
        n = spec.n
        row_ptr = np.ctypeslib.as_array(ctypes.cast(rp, ctypes.POINTER(ctypes.c_int64)), shape=(n + 1,)).copy()
        if m.value:
            col = np.ctypeslib.as_array(ctypes.cast(ci, ctypes.POINTER(ctypes.c_int32)), shape=(m.value,)).copy()
        else:
            col = np.zeros(0, np.int32)
    finally:
        lib.synth_free(rp)
        lib.synth_free(ci)
    return Graph(spec.n, row_ptr, col, spec)


def uniform(count: int, seed: int) -> np.ndarray:
    """U[0,1) FP64 draws, element i from the counter-based stream (seed, i)."""
    lib = _load()
    out = np.empty(count, np.float64)
    if count:
        lib.synth_uniform(count, seed & 0xFFFFFFFFFFFFFFFF, out.ctypes.data)
    return out


def rhs(n: int, k: int, seed: int) -> np.ndarray:
    """Right-hand sides x ~ U(0,1): row-major n x k, drawn in FP64 then rounded
    to FP32 (the GPU's storage type). Both sides use these rounded values."""
    return uniform(n * k, seed).reshape(n, k).astype(np.float32)


def nodes(count: int, n: int, seed: int) -> np.ndarray:
    """`count` node ids uniform in [0, n) (seed nodes of personalized teleports)."""
    lib = _load()
    out = np.empty(count, np.int64)
    if count:
        lib.synth_nodes(count, n, seed & 0xFFFFFFFFFFFFFFFF, out.ctypes.data)
    return out


def dyadic_rhs(n: int, k: int, seed: int, bits: int = 10) -> np.ndarray:
    """x = integer / 2^bits with small integers: every partial sum of such values
    is exact in FP32 and FP64 (as long as the sums stay below 2^24 / 2^bits)."""
    u = uniform(n * k, seed).reshape(n, k)
    return (np.floor(u * 16.0) / float(1 << bits)).astype(np.float32)


def signed_rhs(n: int, k: int, seed: int) -> np.ndarray:
    """x ~ U(-1, 1), row-major n x k, drawn in FP64 and rounded to FP32: signed
    inputs, where sums along reference chains and across columns cancel."""
    return (2.0 * uniform(n * k, seed) - 1.0).reshape(n, k).astype(np.float32)


def wide_rhs(n: int, k: int, seed: int, span: int = 20) -> np.ndarray:
    """Signed x whose magnitudes spread over 2^-span .. 2^span: x = s * m * 2^e
    with s = +-1, m ~ U[1, 2) and e a uniform integer in [-span, span], each
    from its own counter-based draw; rounded to FP32."""
    u = uniform(3 * n * k, seed).reshape(3, n * k)
    s = np.where(u[0] < 0.5, -1.0, 1.0)
    m = 1.0 + u[1]
    e = np.floor(u[2] * (2 * span + 1)).astype(np.int64) - span
    return (s * np.ldexp(m, e)).reshape(n, k).astype(np.float32)


def signed_dyadic_rhs(n: int, k: int, seed: int, bits: int = 10) -> np.ndarray:
    """x = integer / 2^bits with integers in [-16, 15]: signed, and every partial
    sum of such values is exact in FP32 and FP64."""
    u = uniform(n * k, seed).reshape(n, k)
    return ((np.floor(u * 32.0) - 16.0) / float(1 << bits)).astype(np.float32)


def input_kind(kind: str, n: int, k: int, seed: int) -> np.ndarray:
    """Right-hand sides by name: 'uniform' (U(0,1)), 'signed' (U(-1,1)),
    'wide' (signed, magnitudes 2^-20 .. 2^20)."""
    return {"uniform": rhs, "signed": signed_rhs, "wide": wide_rhs}[kind](n, k, seed)


def seed_for(workload: int, graph: int = 0) -> int:
    return BASE_SEED + 1000 * workload + graph


# --- named workloads ------------------------------------------------------
# Workload sizes follow the paper's web/social graph shapes scaled to synthetic
# stand-ins. Calibrated parameters: see the table of achieved values in the
# design notes (m, m/m', m/w').

def tiny_web(seed: int | None = None) -> GraphSpec:
    """n = 10,000, average out-degree ~12, row copy probability 0.7."""
    return GraphSpec(n=10_000, seed=seed_for(1) if seed is None else seed, p_copy=0.7, fidelity=0.97,
                     extra_mean=0.8, fresh_mean=6.0, q_run=0.25, gap_mean=30.0)


def web_862k(seed: int | None = None) -> GraphSpec:
    """n = 862,664, ~19.2 M edges, row copy probability 0.8, high locality."""
    return GraphSpec(n=862_664, seed=seed_for(2) if seed is None else seed, p_copy=0.8, fidelity=0.985,
                     extra_mean=0.35, fresh_mean=17.0, q_run=0.5, gap_mean=24.0)


def web_862k_hc(seed: int | None = None) -> GraphSpec:
    """n = 862,664, ~19 M edges, compressed more than 5x in nnz(A') (Table 1's
    m / m' measure): rows copy a prototype exactly (fidelity 1) with
    probability 0.93 and add few extra successors."""
    return GraphSpec(n=862_664, seed=seed_for(2, 50) if seed is None else seed, p_copy=0.93, fidelity=1.0,
                     extra_mean=0.03, fresh_mean=23.0, q_run=0.5, gap_mean=24.0)


def web_7m4(seed: int | None = None) -> GraphSpec:
    """n = 7.4 M, ~194 M edges (batched personalized PageRank)."""
    return GraphSpec(n=7_400_000, seed=seed_for(3) if seed is None else seed, p_copy=0.8, fidelity=0.985,
                     extra_mean=0.35, fresh_mean=23.0, q_run=0.5, gap_mean=24.0)


def two_region(n: int, seed: int) -> Graph:
    """A 2n x 2n graph whose first n rows link into two regions of ids,
    [0, n) and [n, 2n), the links of each region from its own web-like
    copying-model graph (web_small, seeds seed and seed + 1): a row's
    prototypes in the two regions are drawn independently, so an earlier row
    that matches one part of the row rarely matches the other. The last n
    rows are empty. (A web page's links inside its own site and into a second
    site, copied from different pages.)"""
    g1 = copying_model(web_small(n, seed))
    g2 = copying_model(web_small(n, seed + 1))
    c1, c2 = np.diff(g1.row_ptr), np.diff(g2.row_ptr)
    rp = np.zeros(2 * n + 1, np.int64)
    rp[1:n + 1] = np.cumsum(c1 + c2)
    rp[n + 1:] = rp[n]
    col = np.empty(int(rp[-1]), np.int32)
    start = rp[:n]
    col[np.repeat(start, c1) + (np.arange(g1.m) - np.repeat(g1.row_ptr[:n], c1))] = g1.col
    col[np.repeat(start + c1, c2) + (np.arange(g2.m) - np.repeat(g2.row_ptr[:n], c2))] = g2.col + n
    return Graph(2 * n, rp, col)


def web_small(n: int, seed: int) -> GraphSpec:
    """Web-like graph of n nodes with mean degree ~20 (multi-graph batches,
    warm-start training sets)."""
    return GraphSpec(n=n, seed=seed, p_copy=0.8, fidelity=0.985, extra_mean=0.35, fresh_mean=16.0,
                     q_run=0.5, gap_mean=24.0)


def web_18m5(seed: int | None = None) -> GraphSpec:
    """n = 18.5 M, ~298 M edges (warm-start evaluation)."""
    return GraphSpec(n=18_500_000, seed=seed_for(4) if seed is None else seed, p_copy=0.8, fidelity=0.985,
                     extra_mean=0.3, fresh_mean=10.1, q_run=0.5, gap_mean=24.0)


def web_22m7(seed: int | None = None) -> GraphSpec:
    """n = 22.7 M, ~640 M edges."""
    return GraphSpec(n=22_700_000, seed=seed_for(5) if seed is None else seed, p_copy=0.8, fidelity=0.985,
                     extra_mean=0.4, fresh_mean=24.5, q_run=0.5, gap_mean=24.0)


def social_5m4(seed: int | None = None) -> GraphSpec:
    """n = 5.4 M, ~79 M edges: power-law out-degree (alpha 2.1), row copy
    probability 0.3, uniform random ids (weak locality)."""
    return GraphSpec(n=5_400_000, seed=seed_for(5, 1) if seed is None else seed, p_copy=0.3, fidelity=0.9,
                     extra_mean=2.0, powerlaw=True, alpha=2.1, dmin=2, dmax=200_000, q_run=0.0,
                     gap_mean=24.0, random_ids=True)


def multi_graph_sizes(count: int = 64, lo: float = 1e3, hi: float = 1e6, seed: int | None = None) -> list[int]:
    """Graph sizes log-uniform in [lo, hi]."""
    u = uniform(count, seed_for(3, 500) if seed is None else seed)
    return [int(round(lo * (hi / lo) ** float(v))) for v in u]


def spec_dict(spec: GraphSpec) -> dict:
    return asdict(spec)


__all__ = ["GraphSpec", "Graph", "copying_model", "uniform", "rhs", "nodes", "dyadic_rhs", "signed_rhs", "wide_rhs",
           "signed_dyadic_rhs", "input_kind", "seed_for",
           "tiny_web", "web_862k", "web_862k_hc", "web_7m4", "web_small", "web_18m5", "web_22m7", "social_5m4",
           "multi_graph_sizes", "build", "replace"]

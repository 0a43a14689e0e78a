"""Python binding of libbvg (include/bvg.h): BV-delta adjacency products and
PageRank on GB300.

Argument marshalling only: every step of the products runs in the CUDA
kernels of libbvg.so. PyTorch supplies device memory and streams. The
functions keep the C names. If the library is missing (not built) every call
raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

_lock = threading.Lock()
_lib = None

BVG_OK = 0
BVG_ERR_INVALID_ARG = -1
BVG_ERR_BAD_GRAPH = -2
BVG_ERR_OOM = -3
BVG_ERR_CUDA = -4
BVG_ERR_NOT_CONVERGED = -5
BVG_ERR_NUMERIC = -6
BVG_ERR_TIMEOUT = -7
BVG_ERR_CORRUPT = -8
BVG_ERR_UNSUPPORTED = -9

EXPORTED = [
    "bvg_encode", "bvg_decode", "bvg_stats", "bvg_get_refs", "bvg_host_size", "bvg_upload", "bvg_spmv_Ax",
    "bvg_spmv_xA", "bvg_spmv_xA_host", "bvg_pagerank", "bvg_pagerank_seeds", "bvg_dev_size", "bvg_csr_upload", "bvg_csr_spmv_Ax",
    "bvg_csr_spmv_xA", "bvg_free_host", "bvg_free_dev", "bvg_free_csr", "bvg_status_string", "bvg_last_error",
    "bvg_trace_enable", "bvg_trace_read", "bvg_dev_layout", "bvg_layout_view_get", "bvg_spmv_xA_noalloc",
    "bvg_get_config", "bvg_set_config", "bvg_mlp_create", "bvg_mlp_param_count", "bvg_mlp_set_params",
    "bvg_mlp_get_params", "bvg_features", "bvg_mlp_predict", "bvg_mlp_grad", "bvg_mlp_adam", "bvg_warmstart_train",
    "bvg_warmstart_predict", "bvg_free_mlp", "bvg_batch_create", "bvg_batch_size", "bvg_batch_spmv_xA",
    "bvg_free_batch", "bvg_autotune", "bvg_autotune_info_get", "bvg_autotune_key", "bvg_autotune_cache_lookup",
    "bvg_autotune_cache_store", "bvg_pull_items_size", "bvg_pull_items_fill", "bvg_point_cols_size",
    "bvg_point_cols_fill", "bvg_biclique_encode", "bvg_biclique_stats", "bvg_biclique_get", "bvg_free_biclique",
    "bvg_biclique_gather_lists", "bvg_bitstream_get", "bvg_decode_bits", "bvg_debug_fail_alloc",
    "bvg_device_check", "bvg_csr_cusparse_Ax", "bvg_csr_cusparse_xA", "bvg_biclique_upload",
    "bvg_biclique_spmv_Ax", "bvg_biclique_spmv_xA", "bvg_free_biclique_dev", "bvg_stream_create", "bvg_stream_spmv",
    "bvg_stream_info", "bvg_stream_get_refs", "bvg_free_stream", "bvg_spmv_xA_colblocks", "bvg_spmv_Ax_colblocks",
]


class BvgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64


class EncodeParams(ctypes.Structure):
    _fields_ = [("window", _I32), ("max_chain", _I32), ("min_interval", _I32), ("threads", _I32)]


class GraphStats(ctypes.Structure):
    _fields_ = [("n", _I64), ("m", _I64), ("dropped", _I64), ("added", _I64), ("residual", _I64),
                ("intervals", _I64), ("interval_members", _I64), ("nnz_diff", _I64), ("words", _I64),
                ("rows_with_ref", _I64), ("depth_hist", _I64 * 4), ("bitstream_bits", _I64),
                ("bits_per_edge", ctypes.c_double), ("device_bytes", _I64)]


class LayoutInfo(ctypes.Structure):
    _fields_ = [(f, _I64) for f in ("n", "m", "words", "col_entries", "carry_tiles", "carry_entries",
                                      "structure_bytes", "pull_entries", "pull_items", "pull_intervals",
                                      "tail_items", "point_entries", "point_tail_items")]


class LayoutView(ctypes.Structure):
    _fields_ = [(f, _I64) for f in ("n", "words", "col_entries", "carry_tiles", "carry_entries",
                                      "carry_tile_cols")] + \
               [(f, _P) for f in ("meta", "desc", "rowp", "ent", "colp", "tent", "carry_ptr", "carry", "inv_outdeg")] + \
               [("tail_items", _I64), ("titem_ptr", _P), ("titem", _P)]


class LaunchConfig(ctypes.Structure):
    _fields_ = [("pull_tile", _I32), ("pull_prefix", _I32), ("prefix_min_len", _I32), ("gather_pdl", _I32),
                ("col_block", _I32), ("pull_item", _I32), ("push_points", _I32), ("push_fused", _I32),
                ("pull_fused", _I32)]


class StreamInfo(ctypes.Structure):
    _fields_ = [("n", _I64), ("m", _I64), ("left", _I32), ("pad", _I32), ("blocks", _I64), ("slot_bytes", _I64),
                ("image_bytes", _I64)]


class BicliqueParams(ctypes.Structure):
    _fields_ = [("passes", _I32), ("min_rows", _I32), ("min_cols", _I32), ("pad", _I32), ("seed", ctypes.c_uint64)]


class BicliqueInfo(ctypes.Structure):
    _fields_ = [(f, _I64) for f in ("n", "m", "bicliques", "s_total", "c_total", "residual", "words",
                                      "biclique_edges")]


class AutotuneInfo(ctypes.Structure):
    _fields_ = [("from_cache", _I32), ("candidates", _I32), ("push_us_default", ctypes.c_double),
                ("push_us_best", ctypes.c_double), ("pull_us_default", ctypes.c_double),
                ("pull_us_best", ctypes.c_double)]


class TraceEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", _I64), ("total_ms", ctypes.c_double)]


class PrParams(ctypes.Structure):
    _fields_ = [("damping", ctypes.c_double), ("tol_l1", ctypes.c_double), ("max_iter", _I32), ("dangling", _I32)]


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Loads libbvg.so (building it first if asked and out of date)."""
    global _lib
    if _lib is not None:  # every call goes through here: no lock once loaded
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_needed:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libbvg.so is not built ({_build.LIB}); run __graft_entry__.build()")
        lib = ctypes.CDLL(_build.LIB)
        sig = {
            "bvg_encode": ([_I64, _P, _P, ctypes.POINTER(EncodeParams), ctypes.POINTER(_P)], ctypes.c_int),
            "bvg_decode": ([_P, _P, _P], ctypes.c_int),
            "bvg_stats": ([_P, ctypes.POINTER(GraphStats)], ctypes.c_int),
            "bvg_get_refs": ([_P, _P, _P], ctypes.c_int),
            "bvg_host_size": ([_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)], ctypes.c_int),
            "bvg_upload": ([_P, _P, ctypes.POINTER(_P)], ctypes.c_int),
            "bvg_spmv_Ax": ([_P, _P, _P, _I32, _I64, _P], ctypes.c_int),
            "bvg_spmv_xA": ([_P, _P, _P, _I32, _I64, _P], ctypes.c_int),
            "bvg_spmv_xA_host": ([_P, _P, _P, _I32, _P], ctypes.c_int),
            "bvg_spmv_xA_noalloc": ([_P, _P, _P, _I32, _I64, _P], ctypes.c_int),
            "bvg_pagerank": ([_P, ctypes.POINTER(PrParams), _P, _P, _I32, _P, ctypes.POINTER(_I32),
                              _P, _P], ctypes.c_int),
            "bvg_pagerank_seeds": ([_P, ctypes.POINTER(PrParams), _P, _P, _I32, _P, ctypes.POINTER(_I32),
                                    _P, _P], ctypes.c_int),
            "bvg_dev_size": ([_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)], ctypes.c_int),
            "bvg_csr_upload": ([_I64, _P, _P, _P, ctypes.POINTER(_P)], ctypes.c_int),
            "bvg_csr_spmv_Ax": ([_P, _P, _P, _I32, _I64, _P], ctypes.c_int),
            "bvg_csr_spmv_xA": ([_P, _P, _P, _I32, _I64, _P], ctypes.c_int),
            "bvg_free_host": ([_P], None),
            "bvg_free_dev": ([_P], None),
            "bvg_free_csr": ([_P], None),
            "bvg_status_string": ([ctypes.c_int], ctypes.c_char_p),
            "bvg_last_error": ([], ctypes.c_char_p),
            "bvg_trace_enable": ([_P, ctypes.c_int], ctypes.c_int),
            "bvg_dev_layout": ([_P, ctypes.POINTER(LayoutInfo)], ctypes.c_int),
            "bvg_layout_view_get": ([_P, ctypes.POINTER(LayoutView)], ctypes.c_int),
            "bvg_get_config": ([_P, ctypes.POINTER(LaunchConfig)], ctypes.c_int),
            "bvg_set_config": ([_P, ctypes.POINTER(LaunchConfig)], ctypes.c_int),
            "bvg_trace_read": ([_P, ctypes.POINTER(TraceEntry), _I32, ctypes.POINTER(_I32)], ctypes.c_int),
            "bvg_mlp_create": ([ctypes.c_uint64, ctypes.POINTER(_P)], ctypes.c_int),
            "bvg_mlp_param_count": ([], ctypes.c_int),
            "bvg_mlp_set_params": ([_P, _P, _I64], ctypes.c_int),
            "bvg_mlp_get_params": ([_P, _P, _I64], ctypes.c_int),
            "bvg_features": ([_P, _P, _P], ctypes.c_int),
            "bvg_mlp_predict": ([_P, _P, _I64, _P, _P], ctypes.c_int),
            "bvg_mlp_grad": ([_P, _P, _P, _I64, ctypes.POINTER(ctypes.c_double), _P, _P], ctypes.c_int),
            "bvg_mlp_adam": ([_P, ctypes.c_float, _P], ctypes.c_int),
            "bvg_warmstart_train": ([_P, _P, _P, _I32, _I32, ctypes.c_float, _I64, ctypes.POINTER(ctypes.c_double),
                                     _P], ctypes.c_int),
            "bvg_warmstart_predict": ([_P, _P, _P, _P], ctypes.c_int),
            "bvg_free_mlp": ([_P], None),
            "bvg_batch_create": ([_P, _I32, _P, ctypes.POINTER(_P)], ctypes.c_int),
            "bvg_batch_size": ([_P, ctypes.POINTER(_I32), ctypes.POINTER(_I64), ctypes.POINTER(_I64)], ctypes.c_int),
            "bvg_batch_spmv_xA": ([_P, _P, _P, _I32, _P], ctypes.c_int),
            "bvg_free_batch": ([_P], None),
            "bvg_autotune": ([_P, _I32, ctypes.c_char_p, _P], ctypes.c_int),
            "bvg_autotune_info_get": ([_P, ctypes.POINTER(AutotuneInfo)], ctypes.c_int),
            "bvg_autotune_key": ([_P, _I32, ctypes.c_char_p, _I32], ctypes.c_int),
            "bvg_autotune_cache_lookup": ([ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(LaunchConfig),
                                           ctypes.POINTER(_I32)], ctypes.c_int),
            "bvg_autotune_cache_store": ([ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(LaunchConfig),
                                          ctypes.c_double, ctypes.c_double], ctypes.c_int),
            "bvg_pull_items_size": ([_P, _I32, _I32, ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                                     ctypes.POINTER(_I64)], ctypes.c_int),
            "bvg_pull_items_fill": ([_P, _I32, _I32, _P, _P, _P, _P, _P], ctypes.c_int),
            "bvg_point_cols_size": ([_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)], ctypes.c_int),
            "bvg_point_cols_fill": ([_P, _P, _P, _P, _P], ctypes.c_int),
            "bvg_biclique_encode": ([_I64, _P, _P, ctypes.POINTER(BicliqueParams), ctypes.POINTER(_P)],
                                    ctypes.c_int),
            "bvg_biclique_stats": ([_P, ctypes.POINTER(BicliqueInfo)], ctypes.c_int),
            "bvg_biclique_get": ([_P, _P, _P, _P, _P, _P, _P], ctypes.c_int),
            "bvg_free_biclique": ([_P], None),
            "bvg_biclique_gather_lists": ([_P, _P, _P, _P, _P, _P, _P], ctypes.c_int),
            "bvg_bitstream_get": ([_P, _P, _I64, ctypes.POINTER(_I64)], ctypes.c_int),
            "bvg_decode_bits": ([_I64, _I64, ctypes.POINTER(EncodeParams), _P, _I64, _P, _P], ctypes.c_int),
            "bvg_debug_fail_alloc": ([_I64], ctypes.c_int),
            "bvg_device_check": ([_P, _P], ctypes.c_int),
            "bvg_csr_cusparse_Ax": ([_P, _P, _P, _I32, _I64, _P], ctypes.c_int),
            "bvg_csr_cusparse_xA": ([_P, _P, _P, _I32, _I64, _P], ctypes.c_int),
            "bvg_biclique_upload": ([_P, _P, ctypes.POINTER(_P)], ctypes.c_int),
            "bvg_biclique_spmv_Ax": ([_P, _P, _P, _I32, _I64, _P], ctypes.c_int),
            "bvg_biclique_spmv_xA": ([_P, _P, _P, _I32, _I64, _P], ctypes.c_int),
            "bvg_free_biclique_dev": ([_P], None),
            "bvg_stream_create": ([_I64, _P, _P, _I64, _I32, ctypes.POINTER(EncodeParams), ctypes.POINTER(_P)],
                                  ctypes.c_int),
            "bvg_stream_spmv": ([_P, _P, _P, _I32, _I64, _P], ctypes.c_int),
            "bvg_stream_info": ([_P, ctypes.POINTER(StreamInfo)], ctypes.c_int),
            "bvg_stream_get_refs": ([_P, _P], ctypes.c_int),
            "bvg_free_stream": ([_P], None),
            "bvg_spmv_xA_colblocks": ([_P, _P, _I32, _P, _P, _P, _I32, _I64, _P], ctypes.c_int),
            "bvg_spmv_Ax_colblocks": ([_P, _I32, _P, _P, _P, _I32, _I64, _P], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(rc: int, what: str, allow=()):
    if rc != BVG_OK and rc not in allow:
        lib = load(False)
        raise BvgError(rc, f"{what}: {lib.bvg_status_string(rc).decode()}: {lib.bvg_last_error().decode()}")
    return rc


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class HostGraph:
    """Owns a bvg_host_graph*."""

    def __init__(self, ptr):
        self.ptr = ptr

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.bvg_free_host(self.ptr)
            self.ptr = None


class DevGraph:
    """Owns a bvg_dev_graph*."""

    def __init__(self, ptr, n, m):
        self.ptr, self.n, self.m = ptr, n, m

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.bvg_free_dev(self.ptr)
            self.ptr = None


class CsrGraph:
    def __init__(self, ptr, n, m):
        self.ptr, self.n, self.m = ptr, n, m

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.bvg_free_csr(self.ptr)
            self.ptr = None


class Batch:
    """Owns a bvg_batch* and keeps its graphs alive."""

    def __init__(self, ptr, graphs):
        self.ptr, self.graphs = ptr, list(graphs)
        self.sizes = [g.n for g in graphs]

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.bvg_free_batch(self.ptr)
            self.ptr = None


class Mlp:
    """Owns a bvg_mlp* (the warm-start network)."""

    def __init__(self, ptr):
        self.ptr = ptr

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.bvg_free_mlp(self.ptr)
            self.ptr = None


def _csr_arrays(row_ptr, col):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col, dtype=np.int32)
    return rp, ci, len(rp) - 1


def bvg_encode(row_ptr, col, window=7, max_chain=3, min_interval=4, threads=0) -> HostGraph:
    lib = load()
    rp, ci, n = _csr_arrays(row_ptr, col)
    prm = EncodeParams(window, max_chain, min_interval, threads)
    out = _P()
    _check(lib.bvg_encode(n, rp.ctypes.data, ci.ctypes.data if len(ci) else None, ctypes.byref(prm),
                          ctypes.byref(out)), "bvg_encode")
    return HostGraph(out)


def bvg_host_size(hg: HostGraph):
    n, m = _I64(), _I64()
    _check(load().bvg_host_size(hg.ptr, ctypes.byref(n), ctypes.byref(m)), "bvg_host_size")
    return n.value, m.value


def bvg_decode(hg: HostGraph):
    n, m = bvg_host_size(hg)
    rp = np.empty(n + 1, np.int64)
    ci = np.empty(max(m, 1), np.int32)
    _check(load().bvg_decode(hg.ptr, rp.ctypes.data, ci.ctypes.data), "bvg_decode")
    return rp, ci[:m]


def bvg_bitstream_get(hg: HostGraph):
    """The encoding's bitstream: (uint64 words, number of bits)."""
    nb = _I64()
    lib = load()
    _check(lib.bvg_bitstream_get(hg.ptr, None, 0, ctypes.byref(nb)), "bvg_bitstream_get")
    words = np.zeros(max(1, (nb.value + 63) // 64), np.uint64)
    _check(lib.bvg_bitstream_get(hg.ptr, words.ctypes.data, len(words), ctypes.byref(nb)), "bvg_bitstream_get")
    return words[:(nb.value + 63) // 64], nb.value


def bvg_decode_bits(n: int, m: int, words, nbits: int, window=7, min_interval=4):
    """Decodes a bitstream (uint64 words, MSB first) of n rows and m edges into
    CSR (row_ptr, col)."""
    w = np.ascontiguousarray(words, dtype=np.uint64)
    rp = np.empty(n + 1, np.int64)
    ci = np.empty(max(m, 1), np.int32)
    prm = EncodeParams(window, 0, min_interval, 0)
    _check(load().bvg_decode_bits(n, m, ctypes.byref(prm), w.ctypes.data if len(w) else None, nbits,
                                  rp.ctypes.data, ci.ctypes.data), "bvg_decode_bits")
    return rp, ci[:m]


def bvg_device_check(dg, stream=None) -> None:
    """Raises BvgError(BVG_ERR_TIMEOUT) if a bounded device wait ran out in an
    earlier launch on this graph (synchronises the stream)."""
    _check(load().bvg_device_check(dg.ptr, _stream(stream)), "bvg_device_check")


def bvg_debug_fail_alloc(after: int) -> None:
    """Testing hook: the allocation checkpoint reached after `after` more fails once (-1 disables)."""
    _check(load().bvg_debug_fail_alloc(after), "bvg_debug_fail_alloc")


def bvg_stats(hg: HostGraph) -> dict:
    st = GraphStats()
    _check(load().bvg_stats(hg.ptr, ctypes.byref(st)), "bvg_stats")
    d = {name: getattr(st, name) for name, _ in GraphStats._fields_}
    d["depth_hist"] = list(st.depth_hist)
    return d


def bvg_get_refs(hg: HostGraph):
    n, _ = bvg_host_size(hg)
    ref = np.empty(n, np.int32)
    depth = np.empty(n, np.int32)
    _check(load().bvg_get_refs(hg.ptr, ref.ctypes.data, depth.ctypes.data), "bvg_get_refs")
    return ref, depth


def bvg_upload(hg: HostGraph, stream=None) -> DevGraph:
    lib = load()
    out = _P()
    _check(lib.bvg_upload(hg.ptr, _stream(stream), ctypes.byref(out)), "bvg_upload")
    n, m = _I64(), _I64()
    lib.bvg_dev_size(out, ctypes.byref(n), ctypes.byref(m))
    return DevGraph(out, n.value, m.value)


def _km(t, n):
    """(k, ld) of a row-major n x k tensor (1-D means k = 1)."""
    if t.dim() == 1:
        if t.shape[0] != n or (t.stride(0) != 1 and n > 0):
            raise ValueError("vector must be contiguous with n entries")
        return 1, 1
    if t.dim() == 2 and t.shape[0] == n == 0:  # no rows: any strides
        return t.shape[1], t.shape[1]
    if t.dim() != 2 or t.shape[0] != n or t.stride(1) != 1:
        raise ValueError("expected a row-major n x k tensor")
    return t.shape[1], t.stride(0)


def _fp32_cuda(*ts):
    import torch
    for t in ts:
        if t is None:
            continue
        if t.dtype != torch.float32 or not t.is_cuda:
            raise ValueError("tensors must be float32 CUDA tensors")


def bvg_spmv_Ax(g: DevGraph, x, y, stream=None):
    """y = A x^T on the device (x, y: float32 CUDA tensors, n or n x k)."""
    _fp32_cuda(x, y)
    k, ld = _km(x, g.n)
    if _km(y, g.n) != (k, ld):
        raise ValueError("x and y must have the same shape and strides")
    _check(load().bvg_spmv_Ax(g.ptr, x.data_ptr(), y.data_ptr(), k, ld, _stream(stream)), "bvg_spmv_Ax")
    return y


def bvg_spmv_xA(g: DevGraph, x, y, stream=None):
    """y = x A on the device."""
    _fp32_cuda(x, y)
    k, ld = _km(x, g.n)
    if _km(y, g.n) != (k, ld):
        raise ValueError("x and y must have the same shape and strides")
    _check(load().bvg_spmv_xA(g.ptr, x.data_ptr(), y.data_ptr(), k, ld, _stream(stream)), "bvg_spmv_xA")
    return y


def bvg_spmv_xA_noalloc(g: DevGraph, x, y, stream=None):
    """y = x A using only the library's fixed device scratch (no allocation)."""
    _fp32_cuda(x, y)
    k, ld = _km(x, g.n)
    if _km(y, g.n) != (k, ld):
        raise ValueError("x and y must have the same shape and strides")
    _check(load().bvg_spmv_xA_noalloc(g.ptr, x.data_ptr(), y.data_ptr(), k, ld, _stream(stream)),
           "bvg_spmv_xA_noalloc")
    return y


def bvg_spmv_xA_host(g: DevGraph, x, y, stream=None):
    """y = x A with x, y in host memory (numpy float32 or CPU tensors, n x k contiguous)."""
    def ptr(a):
        if isinstance(a, np.ndarray):
            if a.dtype != np.float32 or not a.flags.c_contiguous:
                raise ValueError("host arrays must be contiguous float32")
            return a.ctypes.data, (a.shape[1] if a.ndim == 2 else 1)
        if a.is_cuda or not a.is_contiguous():
            raise ValueError("host tensors must be contiguous CPU tensors")
        return a.data_ptr(), (a.shape[1] if a.dim() == 2 else 1)
    xp, k = ptr(x)
    yp, k2 = ptr(y)
    if k != k2:
        raise ValueError("x and y must have the same shape")
    _check(load().bvg_spmv_xA_host(g.ptr, xp, yp, k, _stream(stream)), "bvg_spmv_xA_host")
    return y


def bvg_pagerank(g: DevGraph, p0=None, p_init=None, k=1, damping=0.85, tol=1e-8, max_iter=1000, dangling=0,
                 out=None, stream=None):
    """PageRank (Eq. 1) for k teleport vectors. Returns (p, iterations, residuals, status);
    status is BVG_OK or BVG_ERR_NOT_CONVERGED (other failures raise)."""
    import torch
    if p0 is not None:
        _fp32_cuda(p0)
        k = 1 if p0.dim() == 1 else p0.shape[1]
    if out is None:
        out = torch.empty((g.n, k) if k > 1 or (p0 is not None and p0.dim() == 2) else (g.n,),
                          dtype=torch.float32, device="cuda")
    for t in (p0, p_init, out):
        if t is not None and (not t.is_contiguous()):
            raise ValueError("PageRank vectors must be contiguous n x k")
    prm = PrParams(damping, tol, max_iter, dangling)
    iters = _I32()
    resid = np.zeros(k, np.float64)
    rc = load().bvg_pagerank(g.ptr, ctypes.byref(prm), None if p0 is None else p0.data_ptr(),
                             None if p_init is None else p_init.data_ptr(), k, out.data_ptr(), ctypes.byref(iters),
                             resid.ctypes.data, _stream(stream))
    _check(rc, "bvg_pagerank", allow=(BVG_ERR_NOT_CONVERGED,))
    return out, iters.value, resid, rc


def bvg_pagerank_seeds(g: DevGraph, seeds, p_init=None, damping=0.85, tol=1e-8, max_iter=1000, dangling=0,
                       out=None, stream=None):
    """Personalised PageRank (Eq. 1) with one-hot teleport vectors: column c
    teleports to node seeds[c] (k = len(seeds)). Returns (p (n x k),
    iterations, residuals, status) as bvg_pagerank."""
    import torch
    sd = np.ascontiguousarray(np.asarray(seeds, dtype=np.int64).reshape(-1))
    k = int(sd.size)
    if out is None:
        out = torch.empty((g.n, k), dtype=torch.float32, device="cuda")
    for t in (p_init, out):
        if t is not None and (not t.is_contiguous()):
            raise ValueError("PageRank vectors must be contiguous n x k")
    prm = PrParams(damping, tol, max_iter, dangling)
    iters = _I32()
    resid = np.zeros(max(k, 1), np.float64)
    rc = load().bvg_pagerank_seeds(g.ptr, ctypes.byref(prm), sd.ctypes.data if k else None,
                                   None if p_init is None else p_init.data_ptr(), k, out.data_ptr(),
                                   ctypes.byref(iters), resid.ctypes.data, _stream(stream))
    _check(rc, "bvg_pagerank_seeds", allow=(BVG_ERR_NOT_CONVERGED,))
    return out, iters.value, resid[:k], rc


def bvg_csr_upload(row_ptr, col, stream=None) -> CsrGraph:
    lib = load()
    rp, ci, n = _csr_arrays(row_ptr, col)
    out = _P()
    _check(lib.bvg_csr_upload(n, rp.ctypes.data, ci.ctypes.data if len(ci) else None, _stream(stream),
                              ctypes.byref(out)), "bvg_csr_upload")
    return CsrGraph(out, n, int(rp[-1]))


def bvg_csr_spmv_Ax(g: CsrGraph, x, y, stream=None):
    _fp32_cuda(x, y)
    k, ld = _km(x, g.n)
    _check(load().bvg_csr_spmv_Ax(g.ptr, x.data_ptr(), y.data_ptr(), k, ld, _stream(stream)), "bvg_csr_spmv_Ax")
    return y


def bvg_csr_spmv_xA(g: CsrGraph, x, y, stream=None):
    _fp32_cuda(x, y)
    k, ld = _km(x, g.n)
    _check(load().bvg_csr_spmv_xA(g.ptr, x.data_ptr(), y.data_ptr(), k, ld, _stream(stream)), "bvg_csr_spmv_xA")
    return y


def bvg_csr_cusparse_Ax(g: CsrGraph, x, y, stream=None):
    """y = A x^T by cuSPARSE (the vendor-library baseline)."""
    _fp32_cuda(x, y)
    k, ld = _km(x, g.n)
    _check(load().bvg_csr_cusparse_Ax(g.ptr, x.data_ptr(), y.data_ptr(), k, ld, _stream(stream)),
           "bvg_csr_cusparse_Ax")
    return y


def bvg_csr_cusparse_xA(g: CsrGraph, x, y, stream=None):
    """y = x A by cuSPARSE on the CSR of A^T (the vendor-library baseline)."""
    _fp32_cuda(x, y)
    k, ld = _km(x, g.n)
    _check(load().bvg_csr_cusparse_xA(g.ptr, x.data_ptr(), y.data_ptr(), k, ld, _stream(stream)),
           "bvg_csr_cusparse_xA")
    return y


def bvg_layout_view_get(hg: HostGraph) -> dict:
    """Copies of the host-side layout arrays that bvg_upload sends to the GPU."""
    v = LayoutView()
    _check(load().bvg_layout_view_get(hg.ptr, ctypes.byref(v)), "bvg_layout_view_get")

    def arr(ptr, count, ct, dt):
        if count == 0:
            return np.zeros(0, dt)
        return np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(ct)), shape=(count,)).copy()
    n = v.n
    return {
        "n": n, "carry_tile_cols": v.carry_tile_cols,
        "meta": arr(v.meta, n, ctypes.c_uint8, np.uint8),
        "desc": arr(v.desc, n, ctypes.c_uint32, np.uint32),
        "rowp": arr(v.rowp, n + 1, ctypes.c_uint32, np.uint32),
        "ent": arr(v.ent, v.words, ctypes.c_uint32, np.uint32),
        "colp": arr(v.colp, n + 1, ctypes.c_uint32, np.uint32),
        "tent": arr(v.tent, v.col_entries, ctypes.c_uint32, np.uint32),
        "carry_ptr": arr(v.carry_ptr, v.carry_tiles + 1, ctypes.c_uint32, np.uint32),
        "carry": arr(v.carry, v.carry_entries, ctypes.c_uint32, np.uint32),
        "inv_outdeg": arr(v.inv_outdeg, n, ctypes.c_float, np.float32),
        "titem_ptr": arr(v.titem_ptr, n + 1, ctypes.c_uint32, np.uint32),
        "titem": arr(v.titem, v.tail_items, ctypes.c_uint32, np.uint32),
    }


def bvg_dev_layout(g: DevGraph) -> dict:
    info = LayoutInfo()
    _check(load().bvg_dev_layout(g.ptr, ctypes.byref(info)), "bvg_dev_layout")
    return {f: getattr(info, f) for f, _ in LayoutInfo._fields_}


def bvg_get_config(g: DevGraph) -> dict:
    c = LaunchConfig()
    _check(load().bvg_get_config(g.ptr, ctypes.byref(c)), "bvg_get_config")
    return {f: getattr(c, f) for f, _ in LaunchConfig._fields_}


def bvg_set_config(g: DevGraph, **changes) -> dict:
    """Updates fields of the launch configuration; returns the new one."""
    cur = bvg_get_config(g)
    cur.update(changes)
    c = LaunchConfig(**cur)
    _check(load().bvg_set_config(g.ptr, ctypes.byref(c)), "bvg_set_config")
    return cur


def bvg_trace_enable(g: DevGraph, enable: bool = True):
    _check(load().bvg_trace_enable(g.ptr, int(bool(enable))), "bvg_trace_enable")


def bvg_trace_read(g: DevGraph) -> dict:
    """{kernel family: (launches, total ms)} recorded since the last read."""
    buf = (TraceEntry * 32)()
    cnt = _I32()
    _check(load().bvg_trace_read(g.ptr, buf, 32, ctypes.byref(cnt)), "bvg_trace_read")
    return {buf[i].name.decode(): (buf[i].launches, buf[i].total_ms) for i in range(cnt.value)}


def bvg_status_string(status: int) -> str:
    return load().bvg_status_string(status).decode()


# ------------------------------------------------------------ learned warm start

def bvg_mlp_create(seed: int = 0) -> Mlp:
    out = _P()
    _check(load().bvg_mlp_create(int(seed) & (2**64 - 1), ctypes.byref(out)), "bvg_mlp_create")
    return Mlp(out)


def bvg_mlp_set_params(net: Mlp, theta):
    a = np.ascontiguousarray(theta, dtype=np.float32)
    _check(load().bvg_mlp_set_params(net.ptr, a.ctypes.data, a.size), "bvg_mlp_set_params")


def bvg_mlp_get_params(net: Mlp):
    lib = load()
    a = np.zeros(lib.bvg_mlp_param_count(), np.float32)
    _check(lib.bvg_mlp_get_params(net.ptr, a.ctypes.data, a.size), "bvg_mlp_get_params")
    return a


def bvg_features(g: DevGraph, out=None, stream=None):
    """Node features (n x 8 float32 CUDA tensor)."""
    import torch
    if out is None:
        out = torch.empty((g.n, 8), dtype=torch.float32, device="cuda")
    _fp32_cuda(out)
    if tuple(out.shape) != (g.n, 8) or not out.is_contiguous():
        raise ValueError("features: out must be a contiguous n x 8 tensor")
    _check(load().bvg_features(g.ptr, out.data_ptr(), _stream(stream)), "bvg_features")
    return out


def _feat_ok(feat):
    _fp32_cuda(feat)
    if feat.dim() != 2 or feat.shape[1] != 8 or not feat.is_contiguous():
        raise ValueError("features must be a contiguous n x 8 float32 CUDA tensor")


def bvg_mlp_predict(net: Mlp, feat, out=None, stream=None):
    import torch
    _feat_ok(feat)
    n = feat.shape[0]
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device="cuda")
    _fp32_cuda(out)
    _check(load().bvg_mlp_predict(net.ptr, feat.data_ptr(), n, out.data_ptr(), _stream(stream)), "bvg_mlp_predict")
    return out


def bvg_mlp_grad(net: Mlp, feat, target, stream=None):
    """(loss, gradient as a host float32 array) of the mean squared error."""
    _feat_ok(feat)
    _fp32_cuda(target)
    n = feat.shape[0]
    if target.shape != (n,) or not target.is_contiguous():
        raise ValueError("target must be a contiguous vector of n floats")
    lib = load()
    g = np.zeros(lib.bvg_mlp_param_count(), np.float32)
    loss = ctypes.c_double()
    _check(lib.bvg_mlp_grad(net.ptr, feat.data_ptr(), target.data_ptr(), n, ctypes.byref(loss), g.ctypes.data,
                            _stream(stream)), "bvg_mlp_grad")
    return loss.value, g


def bvg_mlp_adam(net: Mlp, lr: float, stream=None):
    _check(load().bvg_mlp_adam(net.ptr, lr, _stream(stream)), "bvg_mlp_adam")


def bvg_warmstart_train(net: Mlp, graphs, p_stars, epochs=20, lr=3e-3, batch=65536, stream=None) -> float:
    """Trains the network on graphs with known PageRank vectors; returns the last pass's mean loss."""
    if len(graphs) != len(p_stars) or not graphs:
        raise ValueError("need one PageRank vector per graph")
    for g, p in zip(graphs, p_stars):
        _fp32_cuda(p)
        if p.shape != (g.n,) or not p.is_contiguous():
            raise ValueError("PageRank vectors must be contiguous with n entries")
    gs = (_P * len(graphs))(*[g.ptr for g in graphs])
    ps = (_P * len(graphs))(*[p.data_ptr() for p in p_stars])
    loss = ctypes.c_double()
    _check(load().bvg_warmstart_train(net.ptr, gs, ps, len(graphs), epochs, lr, batch, ctypes.byref(loss),
                                      _stream(stream)), "bvg_warmstart_train")
    return loss.value


def bvg_warmstart_predict(net: Mlp, g: DevGraph, out=None, stream=None):
    """Starting iterate for bvg_pagerank predicted by the network (n floats, sum 1)."""
    import torch
    if out is None:
        out = torch.empty(g.n, dtype=torch.float32, device="cuda")
    _fp32_cuda(out)
    _check(load().bvg_warmstart_predict(net.ptr, g.ptr, out.data_ptr(), _stream(stream)), "bvg_warmstart_predict")
    return out


# ------------------------------------------------------------ multi-graph batch

def bvg_batch_create(graphs, stream=None) -> Batch:
    graphs = list(graphs)
    arr = (_P * len(graphs))(*[g.ptr for g in graphs])
    out = _P()
    _check(load().bvg_batch_create(arr, len(graphs), _stream(stream), ctypes.byref(out)), "bvg_batch_create")
    return Batch(out, graphs)


def bvg_batch_size(b: Batch):
    c, n, m = _I32(), _I64(), _I64()
    _check(load().bvg_batch_size(b.ptr, ctypes.byref(c), ctypes.byref(n), ctypes.byref(m)), "bvg_batch_size")
    return c.value, n.value, m.value


def bvg_batch_spmv_xA(b: Batch, xs, ys, stream=None):
    """ys[i] = xs[i] A_i for every graph of the batch (float32 CUDA tensors, n_i or n_i x k, contiguous)."""
    if len(xs) != len(b.graphs) or len(ys) != len(b.graphs):
        raise ValueError("one x and one y per graph")
    k = None
    for g, x, y in zip(b.graphs, xs, ys):
        _fp32_cuda(x, y)
        kx, ldx = _km(x, g.n)
        if _km(y, g.n) != (kx, ldx) or ldx != kx:
            raise ValueError("x and y must be contiguous n x k with the same shape")
        if k is None:
            k = kx
        elif k != kx:
            raise ValueError("every graph of a batch takes the same k")
    xa = (_P * len(xs))(*[x.data_ptr() for x in xs])
    ya = (_P * len(ys))(*[y.data_ptr() for y in ys])
    _check(load().bvg_batch_spmv_xA(b.ptr, xa, ya, k, _stream(stream)), "bvg_batch_spmv_xA")
    return ys


# ------------------------------------------------------------------ autotune

def bvg_autotune(g: DevGraph, k: int = 1, cache_path=None, stream=None) -> dict:
    """Times the launch configurations, applies the fastest; returns the config and the timings."""
    path = None if cache_path is None else os.fsencode(cache_path)
    lib = load()
    _check(lib.bvg_autotune(g.ptr, k, path, _stream(stream)), "bvg_autotune")
    info = AutotuneInfo()
    _check(lib.bvg_autotune_info_get(g.ptr, ctypes.byref(info)), "bvg_autotune_info_get")
    out = bvg_get_config(g)
    out.update({f: getattr(info, f) for f, _ in AutotuneInfo._fields_})
    return out


def bvg_autotune_key(g: DevGraph, k: int = 1) -> str:
    buf = ctypes.create_string_buffer(512)
    _check(load().bvg_autotune_key(g.ptr, k, buf, 512), "bvg_autotune_key")
    return buf.value.decode()


def bvg_autotune_cache_lookup(path, key: str):
    """Launch configuration cached under key, or None."""
    c = LaunchConfig()
    found = _I32()
    _check(load().bvg_autotune_cache_lookup(os.fsencode(path), key.encode(), ctypes.byref(c),
                                                 ctypes.byref(found)), "bvg_autotune_cache_lookup")
    return {f: getattr(c, f) for f, _ in LaunchConfig._fields_} if found.value else None


def bvg_autotune_cache_store(path, key: str, config: dict, push_us: float = 0.0, pull_us: float = 0.0):
    c = LaunchConfig(**{f: int(config.get(f, -1) if f in ("push_points", "push_fused", "pull_fused") else config[f])
                        for f, _ in LaunchConfig._fields_})
    _check(load().bvg_autotune_cache_store(os.fsencode(path), key.encode(), ctypes.byref(c), push_us, pull_us),
           "bvg_autotune_cache_store")


def bvg_pull_items(hg: HostGraph, item: int = 8, min_len: int = 32) -> dict:
    """The pull's work items for a host graph (no GPU needed)."""
    lib = load()
    e, k, m = _I64(), _I64(), _I64()
    _check(lib.bvg_pull_items_size(hg.ptr, item, min_len, ctypes.byref(e), ctypes.byref(k), ctypes.byref(m)),
           "bvg_pull_items_size")
    n = bvg_host_size(hg)[0]
    out = {"pent": np.zeros(max(e.value, 1), np.uint32), "istart": np.zeros(k.value + 1, np.uint32),
           "irow": np.zeros(n + 1, np.uint32), "lrow": np.zeros(n + 1, np.uint32),
           "lint": np.zeros(max(2 * m.value, 1), np.uint32)}
    _check(lib.bvg_pull_items_fill(hg.ptr, item, min_len, *[out[f].ctypes.data for f in
                                                            ("pent", "istart", "irow", "lrow", "lint")]),
           "bvg_pull_items_fill")
    out["pent"] = out["pent"][:e.value]
    out["lint"] = out["lint"][:2 * m.value].reshape(-1, 2)
    return out


def bvg_point_cols(hg: HostGraph) -> dict:
    """The push's point columns for a host graph (no GPU needed)."""
    lib = load()
    e, t = _I64(), _I64()
    _check(lib.bvg_point_cols_size(hg.ptr, ctypes.byref(e), ctypes.byref(t)), "bvg_point_cols_size")
    n = bvg_host_size(hg)[0]
    out = {"colp": np.zeros(n + 1, np.uint32), "ent": np.zeros(max(e.value, 1), np.uint32),
           "titem_ptr": np.zeros(n + 1, np.uint32), "titem": np.zeros(max(t.value, 1), np.uint32)}
    _check(lib.bvg_point_cols_fill(hg.ptr, *[out[f].ctypes.data for f in ("colp", "ent", "titem_ptr", "titem")]),
           "bvg_point_cols_fill")
    out["ent"] = out["ent"][:e.value]
    out["titem"] = out["titem"][:t.value]
    return out


def bvg_biclique_encode(row_ptr, col, passes: int = 8, min_rows: int = 2, min_cols: int = 3,
                        seed: int = 0) -> dict:
    """The biclique decomposition of a CSR graph (Sec. 6; host only): the
    arrays s_ptr, s_idx, c_ptr, c_idx, r_ptr, r_col and the sizes."""
    lib = load()
    rp, ci, n = _csr_arrays(row_ptr, col)
    prm = BicliqueParams(passes, min_rows, min_cols, 0, seed)
    h = _P()
    _check(lib.bvg_biclique_encode(n, rp.ctypes.data, ci.ctypes.data, ctypes.byref(prm), ctypes.byref(h)),
           "bvg_biclique_encode")
    try:
        info = BicliqueInfo()
        _check(lib.bvg_biclique_stats(h, ctypes.byref(info)), "bvg_biclique_stats")
        out = {"s_ptr": np.zeros(info.bicliques + 1, np.int64), "s_idx": np.zeros(max(info.s_total, 1), np.int32),
               "c_ptr": np.zeros(info.bicliques + 1, np.int64), "c_idx": np.zeros(max(info.c_total, 1), np.int32),
               "r_ptr": np.zeros(n + 1, np.int64), "r_col": np.zeros(max(info.residual, 1), np.int32)}
        _check(lib.bvg_biclique_get(h, *[out[f].ctypes.data for f in ("s_ptr", "s_idx", "c_ptr", "c_idx", "r_ptr",
                                                                      "r_col")]), "bvg_biclique_get")
        out.update({"row_ptr2": np.zeros(n + 1, np.int64), "row_bic": np.zeros(max(info.s_total, 1), np.int32),
                    "col_ptr2": np.zeros(n + 1, np.int64), "col_bic": np.zeros(max(info.c_total, 1), np.int32),
                    "rt_ptr": np.zeros(n + 1, np.int64), "rt_row": np.zeros(max(info.residual, 1), np.int32)})
        _check(lib.bvg_biclique_gather_lists(h, *[out[f].ctypes.data for f in ("row_ptr2", "row_bic", "col_ptr2",
                                                                               "col_bic", "rt_ptr", "rt_row")]),
               "bvg_biclique_gather_lists")
    finally:
        lib.bvg_free_biclique(h)
    out["s_idx"] = out["s_idx"][:info.s_total]
    out["c_idx"] = out["c_idx"][:info.c_total]
    out["r_col"] = out["r_col"][:info.residual]
    out["row_bic"] = out["row_bic"][:info.s_total]
    out["col_bic"] = out["col_bic"][:info.c_total]
    out["rt_row"] = out["rt_row"][:info.residual]
    out.update({f: getattr(info, f) for f, _ in BicliqueInfo._fields_})
    return out


class BicliqueDev:
    """Device handle of a biclique decomposition (freed with the object)."""

    def __init__(self, ptr, n: int, m: int, info: dict):
        self.ptr, self.n, self.m, self.info = ptr, n, m, info

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.bvg_free_biclique_dev(self.ptr)
            self.ptr = None


def bvg_biclique_upload(row_ptr, col, passes: int = 8, min_rows: int = 2, min_cols: int = 3, seed: int = 0,
                        stream=None) -> BicliqueDev:
    """Decomposes a CSR graph into bicliques and residual edges (Sec. 6, host)
    and copies the decomposition to the current device."""
    lib = load()
    rp, ci, n = _csr_arrays(row_ptr, col)
    prm = BicliqueParams(passes, min_rows, min_cols, 0, seed)
    h = _P()
    _check(lib.bvg_biclique_encode(n, rp.ctypes.data, ci.ctypes.data if len(ci) else None, ctypes.byref(prm),
                                   ctypes.byref(h)), "bvg_biclique_encode")
    try:
        info = BicliqueInfo()
        _check(lib.bvg_biclique_stats(h, ctypes.byref(info)), "bvg_biclique_stats")
        d = _P()
        _check(lib.bvg_biclique_upload(h, _stream(stream), ctypes.byref(d)), "bvg_biclique_upload")
    finally:
        lib.bvg_free_biclique(h)
    return BicliqueDev(d, n, int(rp[-1]), {f: getattr(info, f) for f, _ in BicliqueInfo._fields_})


def bvg_biclique_spmv_Ax(d: BicliqueDev, x, y, stream=None):
    """y = A x^T on the biclique representation (device)."""
    _fp32_cuda(x, y)
    k, ld = _km(x, d.n)
    _check(load().bvg_biclique_spmv_Ax(d.ptr, x.data_ptr(), y.data_ptr(), k, ld, _stream(stream)),
           "bvg_biclique_spmv_Ax")
    return y


def bvg_biclique_spmv_xA(d: BicliqueDev, x, y, stream=None):
    """y = x A on the biclique representation (device)."""
    _fp32_cuda(x, y)
    k, ld = _km(x, d.n)
    _check(load().bvg_biclique_spmv_xA(d.ptr, x.data_ptr(), y.data_ptr(), k, ld, _stream(stream)),
           "bvg_biclique_spmv_xA")
    return y


class Stream:
    """Streamed row blocks (freed with the object)."""

    def __init__(self, ptr, n: int, m: int, left: int):
        self.ptr, self.n, self.m, self.left = ptr, n, m, left

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.bvg_free_stream(self.ptr)
            self.ptr = None


def bvg_stream_create(row_ptr, col, budget_bytes: int, left: bool = False, window=7, max_chain=3,
                      min_interval=4) -> Stream:
    """Row blocks of A (or of A^T for x A) whose images stay in page-locked
    host memory, each at most half of budget_bytes on the device."""
    lib = load()
    rp, ci, n = _csr_arrays(row_ptr, col)
    prm = EncodeParams(window, max_chain, min_interval, 0)
    out = _P()
    _check(lib.bvg_stream_create(n, rp.ctypes.data, ci.ctypes.data if len(ci) else None, int(budget_bytes),
                                 1 if left else 0, ctypes.byref(prm), ctypes.byref(out)), "bvg_stream_create")
    return Stream(out, n, int(rp[-1]), 1 if left else 0)


def bvg_stream_spmv(s: Stream, x, y, stream=None):
    """y = A x^T (or x A for a left stream), the blocks streamed through the device."""
    _fp32_cuda(x, y)
    k, ld = _km(x, s.n)
    if _km(y, s.n) != (k, ld):
        raise ValueError("x and y must have the same shape and strides")
    _check(load().bvg_stream_spmv(s.ptr, x.data_ptr(), y.data_ptr(), k, ld, _stream(stream)), "bvg_stream_spmv")
    return y


def bvg_stream_info(s: Stream) -> dict:
    info = StreamInfo()
    _check(load().bvg_stream_info(s.ptr, ctypes.byref(info)), "bvg_stream_info")
    return {f: getattr(info, f) for f, _ in StreamInfo._fields_ if f != "pad"}


def bvg_stream_get_refs(s: Stream):
    ref = np.empty(s.n, np.int32)
    _check(load().bvg_stream_get_refs(s.ptr, ref.ctypes.data), "bvg_stream_get_refs")
    return ref


# ------------------------------------------------------ column blocks (Sec. 6)

def split_columns(row_ptr, col, cuts):
    """The CSR of A restricted to each column range [cuts[b], cuts[b+1])
    (n rows and the ids unchanged), one (row_ptr, col) per block."""
    rp, ci, n = _csr_arrays(row_ptr, col)
    cuts = np.asarray(cuts, np.int64)
    row_of = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    out = []
    for b in range(len(cuts) - 1):
        sel = (ci >= cuts[b]) & (ci < cuts[b + 1])
        brp = np.zeros(n + 1, np.int64)
        brp[1:] = np.cumsum(np.bincount(row_of[sel], minlength=n))
        out.append((brp, ci[sel].astype(np.int32)))
    return out


class ColumnBlocks:
    """A split into submatrices of consecutive columns, each block encoded
    and uploaded on its own (its own references)."""

    def __init__(self, n: int, cuts, hosts, devs):
        self.n, self.cuts, self.hosts, self.devs = n, np.asarray(cuts, np.int64), hosts, devs
        self._arr = (_P * len(devs))(*[d.ptr for d in devs]) if devs else None

    def stats(self) -> dict:
        """The blocks' encoding statistics, summed."""
        tot = {}
        for h in self.hosts:
            for key, v in bvg_stats(h).items():
                if isinstance(v, (int, float)) and key not in ("n", "bits_per_edge"):
                    tot[key] = tot.get(key, 0) + v
        tot["n"] = self.n
        tot["bits_per_edge"] = tot["bitstream_bits"] / max(tot["m"], 1)
        return tot


def aligned_cuts(n: int, nblocks: int, align: int = 1024):
    """nblocks column ranges of about equal width, inner bounds rounded down
    to multiples of `align` (whole 1024-column tiles let the one-vector x A
    of a block compute just its own columns)."""
    cuts = [0] + [(n * b // nblocks) // align * align for b in range(1, nblocks)] + [n]
    return np.maximum.accumulate(np.asarray(cuts, np.int64))


def bvg_colblocks_create(row_ptr, col, nblocks: int = 2, cuts=None, window=7, max_chain=3, min_interval=4,
                         stream=None, upload: bool = True) -> ColumnBlocks:
    """Splits A at `cuts` (default: aligned_cuts(n, nblocks)), encodes and
    (unless upload is False: host encodings only) uploads each block."""
    rp, ci, n = _csr_arrays(row_ptr, col)
    if cuts is None:
        cuts = aligned_cuts(n, nblocks)
    hosts, devs = [], []
    for brp, bci in split_columns(rp, ci, cuts):
        h = bvg_encode(brp, bci, window=window, max_chain=max_chain, min_interval=min_interval)
        hosts.append(h)
        if upload:
            devs.append(bvg_upload(h, stream=stream))
    return ColumnBlocks(n, cuts, hosts, devs)


def _colblock_args(cb: ColumnBlocks, x, y, scratch):
    import torch
    _fp32_cuda(x, y)
    if not cb.devs:
        raise ValueError("the column blocks were not uploaded")
    k, ld = _km(x, cb.n)
    if _km(y, cb.n) != (k, ld):
        raise ValueError("x and y must have the same shape and strides")
    if scratch is None and len(cb.devs) > 1:
        scratch = torch.empty_like(y)
    return k, ld, scratch


def bvg_spmv_xA_colblocks(cb: ColumnBlocks, x, y, scratch=None, stream=None):
    """y = x A over the column blocks (scratch: like y, allocated if not given)."""
    k, ld, scratch = _colblock_args(cb, x, y, scratch)
    _check(load().bvg_spmv_xA_colblocks(cb._arr, cb.cuts.ctypes.data, len(cb.devs), x.data_ptr(), y.data_ptr(),
                                        scratch.data_ptr() if scratch is not None else None, k, ld,
                                        _stream(stream)), "bvg_spmv_xA_colblocks")
    return y


def bvg_spmv_Ax_colblocks(cb: ColumnBlocks, x, y, scratch=None, stream=None):
    """y = A x^T over the column blocks (scratch: like y, allocated if not given)."""
    k, ld, scratch = _colblock_args(cb, x, y, scratch)
    _check(load().bvg_spmv_Ax_colblocks(cb._arr, len(cb.devs), x.data_ptr(), y.data_ptr(),
                                        scratch.data_ptr() if scratch is not None else None, k, ld,
                                        _stream(stream)), "bvg_spmv_Ax_colblocks")
    return y

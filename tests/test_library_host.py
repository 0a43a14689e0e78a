"""Host-side checks of libbvg (no GPU): the library loads and exports every
symbol include/bvg.h declares; the encoder's reference choice and difference
counts equal the oracle's bit for bit; decode(encode(A)) == A; bad inputs
return the documented status codes."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import synth
import paper_1708_07271_gb300 as bvg
from conftest import ROOT


def header_symbols():
    text = open(os.path.join(ROOT, "include", "bvg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bvg_[A-Za-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol():
    lib = bvg.load()
    syms = header_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(lib, s), s
    assert set(bvg.EXPORTED) <= set(syms)


def graphs():
    yield "tiny_web", synth.copying_model(synth.tiny_web())
    yield "social", synth.copying_model(synth.replace(synth.social_5m4(), n=20_000))
    yield "dense_local", synth.copying_model(synth.GraphSpec(n=3000, seed=5, p_copy=0.9, fidelity=0.9,
                                                             extra_mean=2.0, fresh_mean=40, q_run=0.6,
                                                             gap_mean=3.0))
    rp = np.zeros(101, np.int64)
    yield "empty", synth.Graph(100, rp, np.zeros(0, np.int32))


@pytest.mark.parametrize("name,g", list(graphs()), ids=lambda v: v if isinstance(v, str) else "")
def test_encoder_matches_oracle_and_round_trips(name, g):
    hg = bvg.bvg_encode(g.row_ptr, g.col)
    ref, depth = bvg.bvg_get_refs(hg)
    oref, odepth = oracle.choose_refs(g.row_ptr, g.col)
    np.testing.assert_array_equal(ref, oref)
    np.testing.assert_array_equal(depth, odepth)
    st = bvg.bvg_stats(hg)
    oc = oracle.counts(g.row_ptr, g.col, oref)
    for key in ("dropped", "added", "residual", "intervals", "interval_members", "nnz_diff", "words",
                "rows_with_ref"):
        assert st[key] == oc[key], key
    assert st["n"] == g.n and st["m"] == g.m
    assert sum(st["depth_hist"]) == g.n
    rp, ci = bvg.bvg_decode(hg)
    np.testing.assert_array_equal(rp, g.row_ptr)
    np.testing.assert_array_equal(ci, g.col)


@pytest.mark.parametrize("W,R,L", [(1, 1, 2), (3, 2, 3), (7, 1, 8), (7, 3, 4)])
def test_encoder_parameters(W, R, L):
    g = synth.copying_model(synth.GraphSpec(n=2000, seed=9, p_copy=0.8, fidelity=0.9, extra_mean=1.0,
                                            fresh_mean=10, q_run=0.5, gap_mean=5.0))
    hg = bvg.bvg_encode(g.row_ptr, g.col, window=W, max_chain=R, min_interval=L)
    ref, depth = bvg.bvg_get_refs(hg)
    oref, odepth = oracle.choose_refs(g.row_ptr, g.col, W, R, L)
    np.testing.assert_array_equal(ref, oref)
    assert depth.max() <= R
    rp, ci = bvg.bvg_decode(hg)
    np.testing.assert_array_equal(ci, g.col)


def test_pathological_rows():
    n = 64
    rows = [[] for _ in range(n)]
    rows[0] = list(range(n))                  # full row
    rows[1] = list(range(n))                  # identical copy
    rows[2] = list(range(0, n, 2))            # every other id dropped
    rows[3] = [3]                             # self-loop
    rows[4] = [0, n - 1]                      # first and last ids
    rows[5] = list(range(10, 40))             # one long interval
    rows[6] = list(range(10, 40)) + [n - 1]
    rows[7] = []
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([j for r in rows for j in r], np.int32)
    hg = bvg.bvg_encode(rp, col)
    ref, _ = bvg.bvg_get_refs(hg)
    np.testing.assert_array_equal(ref, oracle.choose_refs(rp, col)[0])
    assert ref[1] == 0
    rp2, ci2 = bvg.bvg_decode(hg)
    np.testing.assert_array_equal(ci2, col)


def test_bad_graphs_rejected():
    rp = np.array([0, 2, 3], np.int64)
    for col in ([1, 0, 1], [0, 0, 1], [0, 5, 1], [0, -1, 1]):
        with pytest.raises(bvg.BvgError) as e:
            bvg.bvg_encode(rp, np.array(col, np.int32))
        assert e.value.status == bvg.BVG_ERR_BAD_GRAPH
    with pytest.raises(bvg.BvgError) as e:
        bvg.bvg_encode(np.array([1, 2, 3], np.int64), np.array([0, 1, 0], np.int32))
    assert e.value.status == bvg.BVG_ERR_BAD_GRAPH
    with pytest.raises(bvg.BvgError) as e:
        bvg.bvg_encode(rp, np.array([0, 1, 1], np.int32), window=8)
    assert e.value.status == bvg.BVG_ERR_UNSUPPORTED


def test_null_arguments():
    lib = bvg.load()
    out = ctypes.c_void_p()
    assert lib.bvg_encode(3, None, None, None, ctypes.byref(out)) == bvg.BVG_ERR_INVALID_ARG
    assert lib.bvg_encode(3, None, None, None, None) == bvg.BVG_ERR_INVALID_ARG
    assert lib.bvg_decode(None, None, None) == bvg.BVG_ERR_INVALID_ARG
    assert lib.bvg_spmv_xA(None, None, None, 1, 1, None) == bvg.BVG_ERR_INVALID_ARG
    assert lib.bvg_spmv_Ax(None, None, None, 1, 1, None) == bvg.BVG_ERR_INVALID_ARG
    assert lib.bvg_pagerank(None, None, None, None, 1, None, None, None, None) == bvg.BVG_ERR_INVALID_ARG
    assert bvg.bvg_status_string(bvg.BVG_ERR_CORRUPT) == "corrupt bitstream"


def test_bits_per_edge_reported():
    g = synth.copying_model(synth.tiny_web())
    st = bvg.bvg_stats(bvg.bvg_encode(g.row_ptr, g.col))
    assert 0 < st["bits_per_edge"] < 32
    assert st["bitstream_bits"] == pytest.approx(st["bits_per_edge"] * st["m"])
    assert st["device_bytes"] > 0

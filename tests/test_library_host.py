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


@pytest.mark.parametrize("W,R,L", [(1, 1, 2), (3, 2, 3), (7, 1, 8), (7, 3, 4), (10, 3, 4), (15, 2, 5), (31, 1, 4)])
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
    for window, max_chain in ((32, 1), (15, 3), (11, 3), (17, 2)):  # window <= 31 and window * max_chain <= 32
        with pytest.raises(bvg.BvgError) as e:
            bvg.bvg_encode(rp, np.array([0, 1, 1], np.int32), window=window, max_chain=max_chain)
        assert e.value.status == bvg.BVG_ERR_UNSUPPORTED
    for window, max_chain in ((8, 3), (10, 3), (16, 2), (31, 1)):
        bvg.bvg_encode(rp, np.array([0, 1, 1], np.int32), window=window, max_chain=max_chain)


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


# ---------------------------------------------------------------- damaged streams, allocation failure
def _stream(name="tiny_web"):
    g = dict(graphs())[name]
    hg = bvg.bvg_encode(g.row_ptr, g.col)
    words, nbits = bvg.bvg_bitstream_get(hg)
    return g, hg, words, nbits


def test_decode_bits_round_trip():
    """The exported bitstream decodes (through the caller-stream decoder) to
    the encoded graph bit for bit."""
    for name in ("tiny_web", "social", "empty"):
        g, hg, words, nbits = _stream(name)
        assert nbits == bvg.bvg_stats(hg)["bitstream_bits"]
        rp, ci = bvg.bvg_decode_bits(g.n, g.m, words, nbits)
        np.testing.assert_array_equal(rp, g.row_ptr)
        np.testing.assert_array_equal(ci, g.col)


def test_truncated_streams_are_corrupt():
    """A stream cut short anywhere (or with extra bits) fails with
    BVG_ERR_CORRUPT."""
    g, hg, words, nbits = _stream()
    rng = np.random.default_rng(1)
    for cut in [nbits - 1, nbits - 7, nbits // 2, 64, 1, 0] + list(rng.integers(1, nbits, 20)):
        # the decoder reads no bit past the stated length
        with pytest.raises(bvg.BvgError) as e:
            bvg.bvg_decode_bits(g.n, g.m, words, int(cut))
        assert e.value.status == bvg.BVG_ERR_CORRUPT, cut
    with pytest.raises(bvg.BvgError) as e:  # the stream followed by one spare bit
        bvg.bvg_decode_bits(g.n, g.m, np.append(words, np.uint64(0)), nbits + 1)
    assert e.value.status == bvg.BVG_ERR_CORRUPT


def test_flipped_bits_are_caught_or_change_the_graph():
    """Single flipped bits: the decoder returns BVG_ERR_CORRUPT or a CSR that
    differs from the original; it never returns the original graph from a
    damaged stream, and never reads or writes outside its buffers. Most flips
    are caught outright."""
    g, hg, words, nbits = _stream()
    rng = np.random.default_rng(2)
    caught = 0
    positions = rng.choice(nbits, 300, replace=False)
    for pos in positions:
        w = words.copy()
        w[pos // 64] ^= np.uint64(1 << (63 - int(pos) % 64))
        try:
            rp, ci = bvg.bvg_decode_bits(g.n, g.m, w, nbits)
        except bvg.BvgError as e:
            assert e.status == bvg.BVG_ERR_CORRUPT, pos
            caught += 1
            continue
        assert not (np.array_equal(rp, g.row_ptr) and np.array_equal(ci, g.col)), pos
    assert caught >= len(positions) // 2, caught


def test_corrupt_stream_edge_cases():
    """Hand-made streams: all zero bits (an endless unary prefix), a reference
    offset past the window, a wrong edge count, a wrong row count."""
    g, hg, words, nbits = _stream()
    with pytest.raises(bvg.BvgError) as e:
        bvg.bvg_decode_bits(g.n, g.m, np.zeros_like(words), nbits)
    assert e.value.status == bvg.BVG_ERR_CORRUPT
    # row 0 written with reference offset 1 (gamma(2) = 010): no earlier row
    with pytest.raises(bvg.BvgError) as e:
        bvg.bvg_decode_bits(2, 0, np.array([np.uint64(0b010 << 61)]), 3)
    assert e.value.status == bvg.BVG_ERR_CORRUPT
    for m in (g.m - 1, g.m + 1):
        with pytest.raises(bvg.BvgError) as e:
            bvg.bvg_decode_bits(g.n, m, words, nbits)
        assert e.value.status == bvg.BVG_ERR_CORRUPT
    with pytest.raises(bvg.BvgError) as e:
        bvg.bvg_decode_bits(g.n - 1, g.m, words, nbits)
    assert e.value.status == bvg.BVG_ERR_CORRUPT


def test_allocation_failure_hook_gives_oom():
    """The allocation-failure hook makes bvg_encode fail with BVG_ERR_OOM
    once; the next call succeeds and encodes the same graph."""
    g = dict(graphs())["tiny_web"]
    bvg.bvg_debug_fail_alloc(0)
    try:
        with pytest.raises(bvg.BvgError) as e:
            bvg.bvg_encode(g.row_ptr, g.col)
        assert e.value.status == bvg.BVG_ERR_OOM
    finally:
        bvg.bvg_debug_fail_alloc(-1)
    hg = bvg.bvg_encode(g.row_ptr, g.col)
    rp, ci = bvg.bvg_decode(hg)
    np.testing.assert_array_equal(ci, g.col)

"""Column blocks (Sec. 6, future work: submatrices of consecutive columns,
so that a reference need only match the part of a row inside one block),
host side: the split partitions A's entries exactly; on a graph whose rows
match different earlier rows in two column ranges, encoding the ranges
separately stores far fewer difference entries (nnz(A')), and on the
single-region web graph it stores about as many."""
import numpy as np
import pytest

import oracle
import synth
import paper_1708_07271_gb300 as bvg


def dense(n, rp, ci):
    d = np.zeros((n, n), np.int8)
    for i in range(n):
        d[i, ci[rp[i]:rp[i + 1]]] = 1
    return d


@pytest.mark.parametrize("cuts", [[0, 300], [0, 150, 300], [0, 1, 299, 300], [0, 100, 100, 300]])
def test_split_partitions_the_entries(cuts):
    g = synth.copying_model(synth.replace(synth.tiny_web(), n=300, seed=31))
    parts = bvg.split_columns(g.row_ptr, g.col, cuts)
    total = sum(dense(g.n, rp, ci).astype(np.int64) for rp, ci in parts)
    np.testing.assert_array_equal(total, dense(g.n, g.row_ptr, g.col))
    for (rp, ci), a, b in zip(parts, cuts[:-1], cuts[1:]):
        assert np.all((ci >= a) & (ci < b)) and rp[-1] == len(ci)
        for i in range(g.n):  # rows stay sorted
            assert np.all(np.diff(ci[rp[i]:rp[i + 1]]) > 0)


def test_blocks_choose_their_own_references():
    """Each block's encoding is the oracle's reference choice on that block."""
    g = synth.two_region(3000, 5)
    for rp, ci in bvg.split_columns(g.row_ptr, g.col, [0, 3000, 6000]):
        ref, depth = bvg.bvg_get_refs(bvg.bvg_encode(rp, ci))
        oref, odepth = oracle.choose_refs(rp, ci)
        np.testing.assert_array_equal(ref, oref)
        np.testing.assert_array_equal(depth, odepth)


def test_two_region_rows_compress_better_in_blocks():
    g = synth.two_region(20_000, 9)
    one = bvg.bvg_colblocks_create(g.row_ptr, g.col, nblocks=1, upload=False).stats()
    two = bvg.bvg_colblocks_create(g.row_ptr, g.col, cuts=[0, 20_000, 40_000], upload=False).stats()
    assert one["m"] == two["m"] == g.m
    assert two["nnz_diff"] < 0.8 * one["nnz_diff"], (two["nnz_diff"], one["nnz_diff"])
    single = synth.copying_model(synth.web_small(40_000, 9))
    a = bvg.bvg_colblocks_create(single.row_ptr, single.col, nblocks=1, upload=False).stats()
    b = bvg.bvg_colblocks_create(single.row_ptr, single.col, nblocks=2, upload=False).stats()
    assert b["nnz_diff"] <= 1.05 * a["nnz_diff"]

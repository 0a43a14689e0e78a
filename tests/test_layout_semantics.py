"""The device layout, read on the CPU: evaluating its entries with the
arithmetic the kernels use (in FP64, in NumPy) must give the oracle's
products. Covers the carry-in lists for every tile size a kernel may use
(a multiple of the carry tile), the interval start/end events, the chain
bits of meta, and the row-major words. No GPU needed."""
import numpy as np
import pytest

import oracle
import synth
import paper_1708_07271_gb300 as bvg

TAG_SHIFT = 30
MASK = (1 << 30) - 1


def chain_weights(L, x):
    """z: x pushed down the reference chains (rows in reverse level order),
    checked against the same weights read from the descendant masks."""
    meta = L["meta"].astype(np.int64)
    off = meta & 31
    depth = meta >> 5
    z = x.astype(np.float64).copy()
    # reverse level order: rows of depth d add into their reference
    for d in range(3, 0, -1):
        rows = np.nonzero((depth == d) & (off > 0))[0]
        np.add.at(z, rows - off[rows], z[rows])
    # the same weights from the descendant masks (what the chain kernel reads)
    zd = x.astype(np.float64).copy()
    desc = L["desc"].astype(np.int64)
    for t in range(32):
        rows = np.nonzero((desc >> t) & 1)[0]
        zd[rows] += x[rows + t + 1]
    np.testing.assert_allclose(zd, z, rtol=1e-12)
    return z


def emulate_xA(L, x, tile):
    n = L["n"]
    z = chain_weights(L, x)
    tent = L["tent"].astype(np.int64)
    tag = tent >> TAG_SHIFT
    src = tent & MASK
    col = np.repeat(np.arange(n), np.diff(L["colp"].astype(np.int64)))
    sign = np.where(tag == 1, -1.0, 1.0)[:, None]
    y = np.zeros_like(z)
    pt = tag < 2
    np.add.at(y, col[pt], sign[pt] * z[src[pt]])
    D = np.zeros_like(z)
    ev = ~pt
    np.add.at(D, col[ev], np.where(tag[ev] == 3, -1.0, 1.0)[:, None] * z[src[ev]])
    G = L["carry_tile_cols"]
    assert tile % G == 0
    for a in range(0, n, tile):
        ct = a // G
        lo, hi = L["carry_ptr"][ct], L["carry_ptr"][ct + 1]
        run = z[L["carry"][lo:hi].astype(np.int64)].sum(axis=0)
        e = min(n, a + tile)
        y[a:e] += run + np.cumsum(D[a:e], axis=0)
    return y


def emulate_Ax(L, x):
    n = L["n"]
    x = x.astype(np.float64)
    c = np.zeros_like(x)
    rowp = L["rowp"].astype(np.int64)
    ent = L["ent"].astype(np.int64)
    for i in range(n):
        w = rowp[i]
        while w < rowp[i + 1]:
            tag, j = ent[w] >> TAG_SHIFT, ent[w] & MASK
            if tag == 0:
                c[i] += x[j]
            elif tag == 1:
                c[i] -= x[j]
            elif tag == 2:
                ln = ent[w + 1] & MASK
                assert ent[w + 1] >> TAG_SHIFT == 3
                c[i] += x[j:j + ln].sum(axis=0)
                w += 1
            w += 1
    y = np.zeros_like(c)
    off = (L["meta"] & 31).astype(np.int64)
    for i in range(n):
        y[i] = c[i] + (y[i - off[i]] if off[i] else 0.0)
    return y


def emulate_Ax_items(L, P, x, item, min_len):
    """The pull as the kernels evaluate it: per work item the sum of its
    signed expanded entries, per row the sum of its items and kept
    intervals, then the chains."""
    n = L["n"]
    x = x.astype(np.float64)
    pent = P["pent"].astype(np.int64)
    sign = np.where(pent >> 31, -1.0, 1.0)[:, None]
    vals = sign * x[pent & 0x7FFFFFFF]
    istart = P["istart"].astype(np.int64)
    sizes = np.diff(istart)
    assert np.all(sizes >= 1) and np.all(sizes <= item)
    part = np.add.reduceat(vals, istart[:-1], axis=0) if len(sizes) else np.zeros((0, x.shape[1]))
    c = np.zeros_like(x)
    irow = P["irow"].astype(np.int64)
    for i in np.nonzero(np.diff(irow))[0]:
        c[i] = part[irow[i]:irow[i + 1]].sum(axis=0)
    lrow = P["lrow"].astype(np.int64)
    assert np.all(P["lint"][:, 1] >= min_len) if len(P["lint"]) else True
    for i in np.nonzero(np.diff(lrow))[0]:
        for s0, ln in P["lint"][lrow[i]:lrow[i + 1]]:
            c[i] += x[s0:s0 + ln].sum(axis=0)
    # every item lies inside its row's entries, rows in order
    rows_of_items = np.repeat(np.arange(n), np.diff(irow))
    assert len(rows_of_items) == len(sizes)
    y = np.zeros_like(c)
    off = (L["meta"] & 31).astype(np.int64)
    for i in range(n):
        y[i] = c[i] + (y[i - off[i]] if off[i] else 0.0)
    return y


GRAPHS = {
    "tiny_web": lambda: synth.copying_model(synth.tiny_web()),
    "ragged": lambda: synth.copying_model(synth.replace(synth.tiny_web(), n=1037, seed=77)),
    "long_runs": lambda: synth.copying_model(synth.GraphSpec(n=3000, seed=6, p_copy=0.6, fidelity=0.95,
                                                             extra_mean=1.0, fresh_mean=300, q_run=0.9,
                                                             run_min=100, run_max=900, gap_mean=50.0)),
    "social": lambda: synth.copying_model(synth.replace(synth.social_5m4(), n=5000)),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_layout_reproduces_products(name):
    g = GRAPHS[name]()
    hg = bvg.bvg_encode(g.row_ptr, g.col)
    L = bvg.bvg_layout_view_get(hg)
    x = synth.rhs(g.n, 2, 3).astype(np.float64)
    want_xA = oracle.csr_xA(g.row_ptr, g.col, x)
    for tile in (128, 256, 1024, 4096):
        np.testing.assert_allclose(emulate_xA(L, x, tile), want_xA, rtol=1e-9, atol=1e-9)
    if g.n <= 5000:
        np.testing.assert_allclose(emulate_Ax(L, x), oracle.csr_Ax(g.row_ptr, g.col, x), rtol=1e-9, atol=1e-9)
    # 1/outdeg and chain bits
    deg = np.diff(g.row_ptr)
    np.testing.assert_array_equal(L["inv_outdeg"], np.where(deg > 0, 1.0 / np.maximum(deg, 1), 0).astype(np.float32))
    ref, depth = bvg.bvg_get_refs(hg)
    off = (L["meta"] & 31).astype(np.int64)
    np.testing.assert_array_equal(np.where(ref >= 0, np.arange(g.n) - ref, 0), off)
    np.testing.assert_array_equal(L["meta"] >> 5, depth)
    desc = np.zeros(g.n, np.int64)
    for i in range(g.n):
        r = ref[i]
        while r >= 0:
            desc[r] |= 1 << (i - r - 1)
            r = ref[r]
    np.testing.assert_array_equal(L["desc"], desc)


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("item,min_len", [(8, 32), (4, 4), (16, 1 << 20), (8, 100)])
def test_pull_items_reproduce_products(name, item, min_len):
    g = GRAPHS[name]()
    hg = bvg.bvg_encode(g.row_ptr, g.col)
    L = bvg.bvg_layout_view_get(hg)
    P = bvg.bvg_pull_items(hg, item, min_len)
    x = synth.rhs(g.n, 2, 4).astype(np.float64)
    np.testing.assert_allclose(emulate_Ax_items(L, P, x, item, min_len), oracle.csr_Ax(g.row_ptr, g.col, x),
                               rtol=1e-9, atol=1e-9)
    # expanded entries count: every single id plus the members of short intervals
    ent = L["ent"].astype(np.int64)
    tag = ent >> TAG_SHIFT
    lens = (ent[np.nonzero(tag == 2)[0] + 1] & MASK)
    assert len(P["pent"]) == int(np.sum(tag < 2) + lens[lens < min_len].sum())
    assert len(P["lint"]) == int(np.sum(lens >= min_len))


@pytest.mark.parametrize("name", list(GRAPHS))
def test_tail_items_cover_the_long_columns(name):
    """The push gather reads a column's first 3 entries itself and its other
    entries through tail items of at most 4: the items must cover exactly
    those entries, column by column, in order."""
    g = GRAPHS[name]()
    L = bvg.bvg_layout_view_get(bvg.bvg_encode(g.row_ptr, g.col))
    colp = L["colp"].astype(np.int64)
    tp = L["titem_ptr"].astype(np.int64)
    items = L["titem"].astype(np.int64)
    assert tp[0] == 0 and tp[-1] == len(items) and np.all(np.diff(tp) >= 0)
    start = items & ((1 << 30) - 1)
    cnt = (items >> 30) + 1
    for j in np.nonzero(np.diff(colp) > 3)[0][:2000]:
        covered = np.concatenate([np.arange(s, s + c) for s, c in zip(start[tp[j]:tp[j + 1]], cnt[tp[j]:tp[j + 1]])])
        np.testing.assert_array_equal(covered, np.arange(colp[j] + 3, colp[j + 1]))
    short = np.diff(colp) <= 3
    assert np.all(np.diff(tp)[short] == 0)


@pytest.mark.parametrize("name", list(GRAPHS))
def test_point_columns_reproduce_products(name):
    """The point columns: y_j = sum over column j's entries of +-z_k must give
    x A; each column lists the nonzeros of column j of A' once, rows in
    increasing order; the tail items cover each column past its first 4."""
    g = GRAPHS[name]()
    hg = bvg.bvg_encode(g.row_ptr, g.col)
    L = bvg.bvg_layout_view_get(hg)
    P = bvg.bvg_point_cols(hg)
    n = g.n
    colp = P["colp"].astype(np.int64)
    ent = P["ent"].astype(np.int64)
    tag, src = ent >> TAG_SHIFT, ent & MASK
    assert colp[0] == 0 and colp[-1] == len(ent) and np.all(np.diff(colp) >= 0)
    assert np.all(tag < 2)
    assert len(ent) == bvg.bvg_stats(hg)["nnz_diff"]  # dropped + added, interval members one by one
    col = np.repeat(np.arange(n), np.diff(colp))
    same = col[1:] == col[:-1]
    assert np.all(src[1:][same] > src[:-1][same])  # rows increase within a column, no repeats
    x = synth.rhs(n, 2, 5).astype(np.float64)
    z = chain_weights(L, x)
    y = np.zeros_like(z)
    np.add.at(y, col, np.where(tag == 1, -1.0, 1.0)[:, None] * z[src])
    np.testing.assert_allclose(y, oracle.csr_xA(g.row_ptr, g.col, x), rtol=1e-9, atol=1e-9)
    tp = P["titem_ptr"].astype(np.int64)
    items = P["titem"].astype(np.int64)
    assert tp[0] == 0 and tp[-1] == len(items)
    start, cnt = items & MASK, (items >> 30) + 1
    assert np.all(cnt <= 4)
    for j in np.nonzero(np.diff(colp) > 4)[0][:2000]:
        covered = np.concatenate([np.arange(s, s + c) for s, c in zip(start[tp[j]:tp[j + 1]], cnt[tp[j]:tp[j + 1]])])
        np.testing.assert_array_equal(covered, np.arange(colp[j] + 4, colp[j + 1]))
    assert np.all(np.diff(tp)[np.diff(colp) <= 4] == 0)


def _csr(rows, n):
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate([np.asarray(r, np.int32) for r in rows]) if rp[-1] else np.zeros(0, np.int32)
    return rp, col


@pytest.mark.parametrize("case", ["no_edges", "one_row", "identical_rows", "full_interval"])
def test_point_columns_edge_cases(case):
    """Point columns of degenerate graphs: no edges, a single row, rows that
    are all copies of their reference (A' nearly empty), and a row that is one
    interval over every id (every member listed once)."""
    n = {"no_edges": 40, "one_row": 1, "identical_rows": 300, "full_interval": 200}[case]
    if case == "no_edges":
        rows = [[] for _ in range(n)]
    elif case == "one_row":
        rows = [[0]]
    elif case == "identical_rows":
        rows = [[3, 17, 18, 19, 20, 21, 250] for _ in range(n)]
    else:
        rows = [list(range(n)) if i == 5 else [i] for i in range(n)]
    rp, col = _csr(rows, n)
    hg = bvg.bvg_encode(rp, col)
    P = bvg.bvg_point_cols(hg)
    L = bvg.bvg_layout_view_get(hg)
    colp = P["colp"].astype(np.int64)
    assert len(colp) == n + 1 and colp[0] == 0 and colp[-1] == len(P["ent"])
    assert len(P["ent"]) == bvg.bvg_stats(hg)["nnz_diff"]
    x = synth.rhs(n, 3, 9).astype(np.float64)
    z = chain_weights(L, x)
    ent = P["ent"].astype(np.int64)
    y = np.zeros_like(z)
    np.add.at(y, np.repeat(np.arange(n), np.diff(colp)), np.where(ent >> TAG_SHIFT == 1, -1.0, 1.0)[:, None]
              * z[ent & MASK])
    np.testing.assert_allclose(y, oracle.csr_xA(rp, col, x), rtol=1e-12, atol=1e-12)
    if case == "identical_rows":  # only the rows without a reference carry entries, all 7 of theirs
        ref, _ = bvg.bvg_get_refs(hg)
        assert len(P["ent"]) == 7 * int(np.sum(ref < 0))

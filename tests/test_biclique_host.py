"""The host biclique extractor (Sec. 6's second compressed format): the
decomposition stores exactly the graph's edges (bicliques and residual
edges disjoint), the oracle's biclique products on it equal the plain CSR
products, it is deterministic, and it finds planted bicliques. No GPU."""
import numpy as np
import pytest

import oracle
import synth
import paper_1708_07271_gb300 as bvg
from oracle import biclique as ob


def csr_edges(g):
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    return np.sort(rows * g.n + g.col.astype(np.int64))


def planted(n=400, seed=3):
    """Sparse random rows plus three planted complete bipartite blocks."""
    rng = np.random.default_rng(seed)
    rows = [set(rng.choice(n, size=int(rng.integers(0, 4)), replace=False).tolist()) for _ in range(n)]
    blocks = [(range(10, 22), range(200, 230)), (range(100, 105), range(0, 60, 3)), (range(300, 340), [7, 8, 9])]
    for s, c in blocks:
        for i in s:
            rows[i].update(c)
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    return synth.Graph(n, rp, np.concatenate([np.array(sorted(r), np.int32) for r in rows]))


GRAPHS = {
    "tiny_web": lambda: synth.copying_model(synth.tiny_web()),
    "social_5000": lambda: synth.copying_model(synth.replace(synth.social_5m4(), n=5000)),
    "planted": planted,
    "no_edges": lambda: synth.Graph(30, np.zeros(31, np.int64), np.zeros(0, np.int32)),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_decomposition_is_exact_and_products_match(name):
    g = GRAPHS[name]()
    dec = bvg.bvg_biclique_encode(g.row_ptr, g.col)
    np.testing.assert_array_equal(ob.edges_of(dec, g.n), csr_edges(g))  # disjoint, nothing lost or added
    assert dec["words"] == ob.words(dec) and dec["biclique_edges"] + dec["residual"] == dec["m"] == len(g.col)
    for r in range(dec["bicliques"]):
        s = dec["s_idx"][dec["s_ptr"][r]:dec["s_ptr"][r + 1]]
        c = dec["c_idx"][dec["c_ptr"][r]:dec["c_ptr"][r + 1]]
        assert len(s) >= 2 and len(c) >= 3 and len(s) * len(c) > len(s) + len(c)  # each one saves words
        assert np.all(np.diff(s) > 0) and np.all(np.diff(c) > 0)
    x = synth.dyadic_rhs(g.n, 3, 11) if g.n else np.zeros((0, 3))
    np.testing.assert_array_equal(ob.biclique_Ax(dec, x), oracle.csr_Ax(g.row_ptr, g.col, x))
    np.testing.assert_array_equal(ob.biclique_xA(dec, x), oracle.csr_xA(g.row_ptr, g.col, x))
    assert dec["words"] <= max(dec["m"], 0)


def test_planted_bicliques_are_found_and_deterministic():
    g = planted()
    a = bvg.bvg_biclique_encode(g.row_ptr, g.col)
    b = bvg.bvg_biclique_encode(g.row_ptr, g.col)
    for f in ("s_ptr", "s_idx", "c_ptr", "c_idx", "r_ptr", "r_col"):
        np.testing.assert_array_equal(a[f], b[f])
    planted_edges = 12 * 30 + 5 * 20 + 40 * 3
    ideal_saving = planted_edges - ((12 + 30) + (5 + 20) + (40 + 3))  # each block as one biclique
    assert a["biclique_edges"] >= 0.9 * planted_edges
    assert a["m"] - a["words"] >= 0.85 * ideal_saving
    cs = {tuple(a["c_idx"][a["c_ptr"][r]:a["c_ptr"][r + 1]]) for r in range(a["bicliques"])}
    assert len(cs) == a["bicliques"]  # bicliques with equal column sets were merged


def test_compression_on_web_and_social_graphs():
    """The biclique format compresses the web-like graph; on the social one
    (copy probability 0.3, random ids) there is little to find."""
    web = synth.copying_model(synth.tiny_web())
    soc = synth.copying_model(synth.replace(synth.social_5m4(), n=5000))
    dw = bvg.bvg_biclique_encode(web.row_ptr, web.col)
    ds = bvg.bvg_biclique_encode(soc.row_ptr, soc.col)
    assert dw["m"] / dw["words"] > 1.5
    assert ds["m"] / ds["words"] >= 1.0


def test_invalid_input():
    rp = np.array([0, 2, 2], np.int64)
    with pytest.raises(bvg.BvgError):
        bvg.bvg_biclique_encode(rp, np.array([1, 0], np.int32))  # row not sorted
    with pytest.raises(bvg.BvgError):
        bvg.bvg_biclique_encode(rp, np.array([0, 5], np.int32))  # id out of range


def segment_sums(ptr, idx, x):
    seg = np.repeat(np.arange(len(ptr) - 1), np.diff(ptr))
    out = np.zeros((len(ptr) - 1,) + x.shape[1:])
    np.add.at(out, seg, x[idx.astype(np.int64)])
    return out


@pytest.mark.parametrize("name", list(GRAPHS))
def test_gather_lists_reproduce_products(name):
    """The lists a device product gathers from, evaluated as the kernels would
    (per-biclique sums, then per-row / per-column gathers of those sums and of
    the residual edges), give the plain products exactly on dyadic inputs."""
    g = GRAPHS[name]()
    d = bvg.bvg_biclique_encode(g.row_ptr, g.col)
    for ptr, lst in (("row_ptr2", "row_bic"), ("col_ptr2", "col_bic"), ("rt_ptr", "rt_row")):
        p, v = d[ptr], d[lst].astype(np.int64)
        assert p[0] == 0 and p[-1] == len(v) and np.all(np.diff(p) >= 0)
        seg = np.repeat(np.arange(g.n), np.diff(p))
        same = seg[1:] == seg[:-1]
        assert np.all(v[1:][same] > v[:-1][same])  # increasing within each list
    x = synth.dyadic_rhs(g.n, 2, 13) if g.n else np.zeros((0, 2))
    c = segment_sums(d["c_ptr"], d["c_idx"], x)     # c_r: sum over C_r
    s = segment_sums(d["s_ptr"], d["s_idx"], x)     # d_r: sum over S_r
    y_ax = segment_sums(d["row_ptr2"], d["row_bic"], c) + segment_sums(d["r_ptr"], d["r_col"], x)
    y_xa = segment_sums(d["col_ptr2"], d["col_bic"], s) + segment_sums(d["rt_ptr"], d["rt_row"], x)
    np.testing.assert_array_equal(y_ax, oracle.csr_Ax(g.row_ptr, g.col, x))
    np.testing.assert_array_equal(y_xa, oracle.csr_xA(g.row_ptr, g.col, x))

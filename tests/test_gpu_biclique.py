"""The biclique-format products (Sec. 6) on the GPU, through the C ABI,
against the oracle's products on the same decomposition (oracle/biclique.py,
the passage's steps in FP64) and against the plain definition, element by
element: |y - y*| <= 1e-5 * max(|y*|, s), s = (|x| A)_j or (A |x|)_i (the
format has only +1 entries: s is the magnitude of the terms). Dyadic inputs
are exact and must match bit for bit."""
import numpy as np
import pytest

import oracle
import oracle.biclique as obic
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1708_07271_gb300 as bvg  # noqa: E402

RTOL = 1e-5

GRAPHS = {
    "tiny_web": lambda: synth.copying_model(synth.tiny_web()),
    "social_20k": lambda: synth.copying_model(synth.replace(synth.social_5m4(), n=20_000)),
    "ragged_1037": lambda: synth.copying_model(synth.replace(synth.tiny_web(), n=1037, seed=77)),
    "empty_rows": lambda: synth.Graph(64, np.zeros(65, np.int64), np.zeros(0, np.int32)),
    "hubs": lambda: hub_graph(),
}


def hub_graph():
    """Rows and columns with thousands of entries: rows 3 and 2999 hold every
    id, column 17 every row, and rows 100..199 share one long block of
    columns (a biclique with a large C)."""
    g = synth.copying_model(synth.replace(synth.tiny_web(), n=3000, seed=12))
    rows = []
    for i in range(g.n):
        r = set(g.col[g.row_ptr[i]:g.row_ptr[i + 1]].tolist()) | {17}
        if i in (3, 2999):
            r |= set(range(g.n))
        if 100 <= i < 200:
            r |= set(range(500, 2900))
        rows.append(np.array(sorted(r), np.int32))
    rp = np.zeros(g.n + 1, np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    return synth.Graph(g.n, rp, np.concatenate(rows))
_cache = {}


def graph(name):
    if name not in _cache:
        g = GRAPHS[name]()
        dec = bvg.bvg_biclique_encode(g.row_ptr, g.col)
        _cache[name] = (g, dec, bvg.bvg_biclique_upload(g.row_ptr, g.col))
    return _cache[name]


def check(got, want, mag, what):
    err = np.abs(got.astype(np.float64) - want)
    bad = ~(err <= RTOL * np.maximum(np.abs(want), mag) + 1e-300)
    assert not bad.any(), f"{what}: {int(bad.sum())} entries off, worst {err.max():.3e}"


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("k", [1, 2, 8, 33])
def test_biclique_products_match_oracle(name, k):
    g, dec, d = graph(name)
    if name != "empty_rows":
        assert d.info["bicliques"] > 0
    x = synth.rhs(g.n, k, synth.seed_for(9, k))
    x64 = x.astype(np.float64)
    xt = torch.from_numpy(x).cuda()
    y = torch.full_like(xt, float("nan"))
    bvg.bvg_biclique_spmv_Ax(d, xt, y)
    got = y.cpu().numpy()
    mag = oracle.csr_Ax(g.row_ptr, g.col, np.abs(x64))
    check(got, obic.biclique_Ax(dec, x64), mag, f"Ax vs the passage's steps {name} k={k}")
    check(got, oracle.csr_Ax(g.row_ptr, g.col, x64), mag, f"Ax vs the definition {name} k={k}")
    y.fill_(float("nan"))
    bvg.bvg_biclique_spmv_xA(d, xt, y)
    got = y.cpu().numpy()
    mag = oracle.csr_xA(g.row_ptr, g.col, np.abs(x64))
    check(got, obic.biclique_xA(dec, x64), mag, f"xA vs the passage's steps {name} k={k}")
    check(got, oracle.csr_xA(g.row_ptr, g.col, x64), mag, f"xA vs the definition {name} k={k}")


@pytest.mark.parametrize("name", ["tiny_web", "social_20k"])
def test_biclique_signed_dyadic_bit_exact_and_deterministic(name):
    g, dec, d = graph(name)
    for k in (1, 4, 32):
        x = synth.signed_dyadic_rhs(g.n, k, synth.seed_for(9, 50 + k))
        xt = torch.from_numpy(x).cuda()
        y = torch.empty_like(xt)
        bvg.bvg_biclique_spmv_Ax(d, xt, y)
        np.testing.assert_array_equal(y.cpu().numpy().astype(np.float64), oracle.csr_Ax(g.row_ptr, g.col, x))
        bvg.bvg_biclique_spmv_xA(d, xt, y)
        y2 = torch.empty_like(xt)
        bvg.bvg_biclique_spmv_xA(d, xt, y2)
        assert torch.equal(y, y2)
        np.testing.assert_array_equal(y.cpu().numpy().astype(np.float64), oracle.csr_xA(g.row_ptr, g.col, x))


def test_biclique_signed_and_wide_inputs():
    g, dec, d = graph("tiny_web")
    for kind in ("signed", "wide"):
        x = synth.input_kind(kind, g.n, 3, synth.seed_for(9, 70))
        x64 = x.astype(np.float64)
        xt = torch.from_numpy(x).cuda()
        y = torch.empty_like(xt)
        bvg.bvg_biclique_spmv_Ax(d, xt, y)
        check(y.cpu().numpy(), oracle.csr_Ax(g.row_ptr, g.col, x64), oracle.csr_Ax(g.row_ptr, g.col, np.abs(x64)),
              f"Ax {kind}")
        bvg.bvg_biclique_spmv_xA(d, xt, y)
        check(y.cpu().numpy(), oracle.csr_xA(g.row_ptr, g.col, x64), oracle.csr_xA(g.row_ptr, g.col, np.abs(x64)),
              f"xA {kind}")


def test_biclique_invalid_arguments():
    g, dec, d = graph("tiny_web")
    x = torch.ones(g.n, device="cuda")
    with pytest.raises(bvg.BvgError) as e:
        bvg.bvg_biclique_spmv_xA(d, x, x)
    assert e.value.status == bvg.BVG_ERR_INVALID_ARG

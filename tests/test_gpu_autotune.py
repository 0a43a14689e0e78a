"""Autotuner on the GPU: the chosen configuration is one of the candidates,
products under it still match the oracle (product tolerance 1e-5 of the
magnitude the compressed formula touches), the cache file gives the same
choice to a fresh upload of the same graph without a search, and the
bvg_get_config view reflects it."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1708_07271_gb300 as bvg  # noqa: E402


def check(g, ref, dg, k):
    x = synth.rhs(g.n, k, synth.seed_for(50, k))
    x64 = x.astype(np.float64)
    xt = torch.from_numpy(x).cuda()
    y = torch.full_like(xt, float("nan"))
    bvg.bvg_spmv_xA(dg, xt, y)
    want, mag = oracle.csr_xA(g.row_ptr, g.col, x64), oracle.bv_xA(g.row_ptr, g.col, ref, x64, absval=True)
    assert np.all(np.abs(y.cpu().numpy() - want) <= 1e-5 * np.maximum(np.abs(want), mag))
    y.fill_(float("nan"))
    bvg.bvg_spmv_Ax(dg, xt, y)
    want, mag = oracle.csr_Ax(g.row_ptr, g.col, x64), oracle.bv_Ax(g.row_ptr, g.col, ref, x64, absval=True)
    assert np.all(np.abs(y.cpu().numpy() - want) <= 1e-5 * np.maximum(np.abs(want), mag))


@pytest.mark.parametrize("k", [1, 8, 32])
def test_autotune_and_cache(tmp_path, k):
    spec = synth.replace(synth.web_small(30_000, synth.seed_for(51)), n=30_000)
    g = synth.copying_model(spec)
    hg = bvg.bvg_encode(g.row_ptr, g.col)
    ref, _ = bvg.bvg_get_refs(hg)
    dg = bvg.bvg_upload(hg)
    path = tmp_path / "tune.json"
    res = bvg.bvg_autotune(dg, k, path)
    assert res["from_cache"] == 0 and res["candidates"] > 0
    assert res["pull_tile"] in (128, 256, 512, 1024) and res["gather_pdl"] in (0, 1)
    assert res["col_block"] <= max(1, k) and res["push_us_best"] > 0 and res["pull_us_best"] > 0
    if k == 1:  # the graph's row tiles fit the one-launch pull: the search chose between the two pulls
        assert res["pull_fused"] in (0, 1)
    check(g, ref, dg, k)
    key = bvg.bvg_autotune_key(dg, k)
    assert key.endswith(f"/k{k}")
    cached = bvg.bvg_autotune_cache_lookup(path, key)
    assert cached == {f: res[f] for f in cached}
    dg2 = bvg.bvg_upload(hg)  # same layout: same key, no search
    res2 = bvg.bvg_autotune(dg2, k, path)
    assert res2["from_cache"] == 1 and res2["candidates"] == 0
    assert {f: res2[f] for f in cached} == cached
    check(g, ref, dg2, k)

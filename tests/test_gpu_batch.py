"""Multi-graph batch: every graph's product from one pair of launches equals
the one-graph product bit for bit (same per-tile code, same column blocks and
vector widths), and the oracle within the product tolerance (1e-5 of the
magnitude the compressed formula touches)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1708_07271_gb300 as bvg  # noqa: E402

RTOL = 1e-5
_cache = {}


def batch_graphs():
    """Sizes log-uniform in [1e3, 1e5] plus edge cases: one row, a ragged
    size just past a tile, an empty graph, and a social-shaped graph."""
    if "graphs" not in _cache:
        sizes = synth.multi_graph_sizes(count=12, lo=1e3, hi=1e5, seed=synth.seed_for(30))
        specs = [synth.web_small(int(n), synth.seed_for(30, i)) for i, n in enumerate(sizes)]
        specs += [synth.replace(synth.tiny_web(), n=1, seed=3), synth.replace(synth.tiny_web(), n=1025, seed=4),
                  synth.replace(synth.social_5m4(), n=5000, seed=5)]
        out = []
        for spec in specs:
            g = synth.copying_model(spec)
            hg = bvg.bvg_encode(g.row_ptr, g.col)
            ref, _ = bvg.bvg_get_refs(hg)
            out.append((g, bvg.bvg_upload(hg), ref))
        empty = bvg.bvg_encode(np.zeros(1, np.int64), np.zeros(0, np.int32))
        out.insert(5, (None, bvg.bvg_upload(empty), None))
        _cache["graphs"] = out
    return _cache["graphs"]


@pytest.mark.parametrize("k", [1, 2, 4, 7, 32, 40])
def test_batch_matches_single_and_oracle(k):
    items = batch_graphs()
    dgs = [d for _, d, _ in items]
    b = bvg.bvg_batch_create(dgs)
    count, total_n, total_m = bvg.bvg_batch_size(b)
    assert count == len(items) and total_n == sum(d.n for d in dgs)
    xs, ys, ys1 = [], [], []
    for i, (g, d, _) in enumerate(items):
        x = torch.from_numpy(synth.rhs(max(d.n, 0), k, synth.seed_for(31, i))).cuda()
        if k == 1:
            x = x.reshape(-1)
        xs.append(x)
        ys.append(torch.full_like(x, float("nan")))
        ys1.append(torch.full_like(x, float("nan")))
    for _ in range(2):  # the second call replays the captured CUDA graph
        for y in ys:
            y.fill_(float("nan"))
        bvg.bvg_batch_spmv_xA(b, xs, ys)
        torch.cuda.synchronize()
        for (g, d, ref), x, y, y1 in zip(items, xs, ys, ys1):
            if d.n == 0:
                continue
            bvg.bvg_spmv_xA(d, x, y1)
            assert torch.equal(y, y1), "batch result differs from the one-graph product"
            x64 = x.cpu().numpy().astype(np.float64).reshape(d.n, -1)
            want = oracle.csr_xA(g.row_ptr, g.col, x64)
            mag = oracle.bv_xA(g.row_ptr, g.col, ref, x64, absval=True)
            got = y.cpu().numpy().astype(np.float64).reshape(d.n, -1)
            err = np.abs(got - want)
            assert np.all(err <= RTOL * np.maximum(np.abs(want), mag) + 1e-30), err.max()


def test_batch_new_buffers_and_invalid_args():
    items = batch_graphs()
    dgs = [d for _, d, _ in items]
    b = bvg.bvg_batch_create(dgs)
    xs = [torch.rand(max(d.n, 1), device="cuda")[: d.n] for d in dgs]
    ys = [torch.empty(d.n, device="cuda") for d in dgs]
    bvg.bvg_batch_spmv_xA(b, xs, ys)
    ys2 = [torch.empty(d.n, device="cuda") for d in dgs]  # other buffers: the table is re-staged
    bvg.bvg_batch_spmv_xA(b, xs, ys2)
    torch.cuda.synchronize()
    for y, y2 in zip(ys, ys2):
        assert torch.equal(y, y2)
    with pytest.raises(ValueError):
        bvg.bvg_batch_spmv_xA(b, xs[:-1], ys[:-1])
    with pytest.raises(bvg.BvgError):
        bvg.bvg_batch_create([])

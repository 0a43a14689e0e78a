"""Personalised PageRank with one-hot teleport vectors given by their nodes
(Eq. 1 with p0 = [e_s1, ..., e_sk]) through bvg_pagerank_seeds, against the
FP64 oracle (L1 <= 1e-6 per column, as the other PageRank tests) and against
bvg_pagerank on the same vectors written out densely: the updates do the same
arithmetic on the same values, so the iterations match and the iterates
agree to the last few units in the last place (at k >= 2 the order in which
a CTA adds its tiles' sums varies between runs)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1708_07271_gb300 as bvg  # noqa: E402

_cache = {}


def graph(name):
    if name not in _cache:
        g = {"tiny_web": lambda: synth.copying_model(synth.tiny_web()),
             "social_20k": lambda: synth.copying_model(synth.replace(synth.social_5m4(), n=20_000)),
             "web_862k": lambda: synth.copying_model(synth.web_862k())}[name]()
        _cache[name] = (g, bvg.bvg_upload(bvg.bvg_encode(g.row_ptr, g.col)))
    return _cache[name]


def l1(a, b):
    return float(np.abs(np.asarray(a, np.float64).reshape(-1) - np.asarray(b, np.float64).reshape(-1)).sum())


def dense(seeds, n):
    P0 = np.zeros((n, len(seeds)), np.float32)
    P0[np.asarray(seeds), np.arange(len(seeds))] = 1.0
    return P0


@pytest.mark.parametrize("name", ["tiny_web", "social_20k"])
@pytest.mark.parametrize("k", [1, 2, 8, 32])
@pytest.mark.parametrize("dangling", [0, 1])
def test_seeds_match_oracle_and_dense_teleport(name, k, dangling):
    g, dg = graph(name)
    seeds = synth.nodes(k, g.n, 400 + k)
    P0 = dense(seeds, g.n)
    p, it, res, rc = bvg.bvg_pagerank_seeds(dg, seeds, tol=1e-8, max_iter=500, dangling=dangling)
    assert rc == bvg.BVG_OK and (res < 1e-8).all(), (rc, it, res)
    got = p.cpu().numpy()
    want, _, _ = oracle.pagerank(g.row_ptr, g.col, alpha=0.15, p0=P0.astype(np.float64), tol=1e-13,
                                 max_iter=2000, dangling=dangling)
    for c in range(k):
        assert l1(got[:, c], want[:, c]) <= 1e-6, c
    pd, itd, _, rcd = bvg.bvg_pagerank(dg, p0=torch.from_numpy(P0).cuda(), tol=1e-8, max_iter=500,
                                       dangling=dangling)
    assert rcd == rc and itd == it
    ref = pd.cpu().numpy().reshape(g.n, k)
    if k == 1:
        np.testing.assert_array_equal(got, ref)  # the same dense vector, the same kernels
    else:
        for c in range(k):
            assert l1(got[:, c], ref[:, c]) <= 1e-7, c


def test_seeds_fixed_count_and_start():
    """A fixed number of updates (not converged) from a given start, and a
    repeated seed (two identical columns)."""
    g, dg = graph("tiny_web")
    seeds = np.array([5, 17, 17, g.n - 1], np.int64)
    P0 = dense(seeds, g.n).astype(np.float64)
    start = torch.full((g.n, 4), 1.0 / g.n, device="cuda")
    p, it, res, rc = bvg.bvg_pagerank_seeds(dg, seeds, p_init=start, tol=1e-12, max_iter=3)
    assert rc == bvg.BVG_ERR_NOT_CONVERGED and it == 3
    want, _, _ = oracle.pagerank(g.row_ptr, g.col, alpha=0.15, p0=P0, p_init=np.full((g.n, 4), 1.0 / g.n),
                                 tol=0.0, max_iter=3)
    got = p.cpu().numpy()
    for c in range(4):
        assert l1(got[:, c], want[:, c]) <= 1e-6, c
    assert np.array_equal(got[:, 1], got[:, 2])


def test_seeds_rejected_before_any_launch():
    g, dg = graph("tiny_web")
    for bad in ([-1, 0], [0, g.n], [3, 1 << 40]):
        with pytest.raises(bvg.BvgError, match="outside"):
            bvg.bvg_pagerank_seeds(dg, bad)
    with pytest.raises(bvg.BvgError):
        bvg.bvg_pagerank_seeds(dg, [1, 2, 3])  # k = 3 is not a supported width
    p, it, res, rc = bvg.bvg_pagerank_seeds(dg, [0, 1], tol=1e-8, max_iter=500)  # the handle still works
    assert rc == bvg.BVG_OK
    bvg.bvg_device_check(dg)


def test_seeds_full_size_k32():
    """n = 862,664, 32 seeds: the same updates as the dense one-hot vectors."""
    g, dg = graph("web_862k")
    seeds = synth.nodes(32, g.n, synth.seed_for(3, 2))
    p, it, res, rc = bvg.bvg_pagerank_seeds(dg, seeds, tol=1e-8, max_iter=1000)
    assert rc == bvg.BVG_OK and (res < 1e-8).all(), (rc, it, res)
    pd, itd, _, _ = bvg.bvg_pagerank(dg, p0=torch.from_numpy(dense(seeds, g.n)).cuda(), tol=1e-8, max_iter=1000)
    assert itd == it
    got, ref = p.cpu().numpy(), pd.cpu().numpy()
    for c in range(32):
        assert l1(got[:, c], ref[:, c]) <= 1e-7, c
        assert abs(float(got[:, c].astype(np.float64).sum()) - 1.0) < 1e-5

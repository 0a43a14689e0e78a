"""GPU parity: the CUDA path through the C ABI against the CPU oracle,
element by element.

Tolerance for a product entry (derived from the arithmetic): FP32 values with
compensated sums give |y - y*| <= ~2^-23 * (sum of the magnitudes of the
terms the compressed formula adds); the test allows 1e-5 of
max(|y*|, s) where s is that magnitude, computed by the oracle on its own
difference rows. Dyadic inputs make every partial sum exact in FP32, so
there the results must match bit for bit. PageRank: L1 distance to the
oracle <= 1e-6.
"""
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


def encode(g):
    hg = bvg.bvg_encode(g.row_ptr, g.col)
    ref, _ = bvg.bvg_get_refs(hg)
    return hg, bvg.bvg_upload(hg), ref


def check_close(got, want, mag, what):
    err = np.abs(got.astype(np.float64) - want)
    bound = RTOL * np.maximum(np.abs(want), mag) + 1e-30
    bad = np.nonzero(~(err <= bound))  # NaN (an entry never written) counts as a mismatch
    assert bad[0].size == 0, f"{what}: {bad[0].size} entries off, worst {err.max():.3e} at {np.argmax(err)}"


GRAPHS = {
    "tiny_web": lambda: synth.copying_model(synth.tiny_web()),
    "ragged_1037": lambda: synth.copying_model(synth.replace(synth.tiny_web(), n=1037, seed=77)),
    "social_20k": lambda: synth.copying_model(synth.replace(synth.social_5m4(), n=20_000)),
    "dense_local": lambda: synth.copying_model(synth.GraphSpec(n=3000, seed=5, p_copy=0.9, fidelity=0.9,
                                                               extra_mean=2.0, fresh_mean=40, q_run=0.6,
                                                               gap_mean=3.0)),
    "long_runs": lambda: synth.copying_model(synth.GraphSpec(n=5000, seed=6, p_copy=0.6, fidelity=0.95,
                                                             extra_mean=1.0, fresh_mean=300, q_run=0.9,
                                                             run_min=100, run_max=900, gap_mean=50.0)),
}
_cache = {}


def graph(name):
    if name not in _cache:
        g = GRAPHS[name]()
        _cache[name] = (g, *encode(g))
    return _cache[name]


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("k", [1, 2, 7, 8, 32, 33])
def test_products_match_oracle(name, k):
    g, hg, dg, ref = graph(name)
    x = synth.rhs(g.n, k, synth.seed_for(1, 100 + k))
    x64 = x.astype(np.float64)
    xt = torch.from_numpy(x).cuda()
    y = torch.full_like(xt, float("nan"))
    bvg.bvg_spmv_xA(dg, xt, y)
    check_close(y.cpu().numpy(), oracle.csr_xA(g.row_ptr, g.col, x64),
                oracle.bv_xA(g.row_ptr, g.col, ref, x64, absval=True), f"xA {name} k={k}")
    y.fill_(float("nan"))
    bvg.bvg_spmv_Ax(dg, xt, y)
    check_close(y.cpu().numpy(), oracle.csr_Ax(g.row_ptr, g.col, x64),
                oracle.bv_Ax(g.row_ptr, g.col, ref, x64, absval=True), f"Ax {name} k={k}")


@pytest.mark.parametrize("name", ["tiny_web", "social_20k", "long_runs"])
@pytest.mark.parametrize("k", [1, 4, 32])
def test_dyadic_inputs_bit_exact(name, k):
    g, hg, dg, ref = graph(name)
    x = synth.dyadic_rhs(g.n, k, synth.seed_for(1, 200 + k))
    xt = torch.from_numpy(x).cuda()
    y = torch.empty_like(xt)
    bvg.bvg_spmv_xA(dg, xt, y)
    np.testing.assert_array_equal(y.cpu().numpy().astype(np.float64), oracle.csr_xA(g.row_ptr, g.col, x))
    bvg.bvg_spmv_Ax(dg, xt, y)
    np.testing.assert_array_equal(y.cpu().numpy().astype(np.float64), oracle.csr_Ax(g.row_ptr, g.col, x))


def test_strided_and_unaligned_views():
    g, hg, dg, ref = graph("tiny_web")
    base = torch.from_numpy(synth.rhs(g.n, 11, 5)).cuda()
    x = base[:, 1:6]  # ld = 11, misaligned start: scalar loads
    y_full = torch.zeros(g.n, 11, device="cuda")
    y = y_full[:, 3:8]
    bvg.bvg_spmv_xA(dg, x, y)
    x64 = x.cpu().numpy().astype(np.float64)
    check_close(y.cpu().numpy(), oracle.csr_xA(g.row_ptr, g.col, x64),
                oracle.bv_xA(g.row_ptr, g.col, ref, x64, absval=True), "strided xA")
    assert (y_full[:, :3] == 0).all() and (y_full[:, 8:] == 0).all()


def test_deterministic():
    g, hg, dg, ref = graph("tiny_web")
    xt = torch.from_numpy(synth.rhs(g.n, 8, 3)).cuda()
    y1, y2 = torch.empty_like(xt), torch.empty_like(xt)
    bvg.bvg_spmv_xA(dg, xt, y1)
    bvg.bvg_spmv_xA(dg, xt, y2)
    assert torch.equal(y1, y2)


def test_csr_baseline_matches_oracle():
    g, hg, dg, ref = graph("tiny_web")
    cg = bvg.bvg_csr_upload(g.row_ptr, g.col)
    for k in (1, 8, 33):
        x = synth.rhs(g.n, k, 9 + k)
        x64 = x.astype(np.float64)
        xt = torch.from_numpy(x).cuda()
        y = torch.empty_like(xt)
        bvg.bvg_csr_spmv_xA(cg, xt, y)
        np.testing.assert_allclose(y.cpu().numpy(), oracle.csr_xA(g.row_ptr, g.col, x64), rtol=1e-5)
        bvg.bvg_csr_spmv_Ax(cg, xt, y)
        np.testing.assert_allclose(y.cpu().numpy(), oracle.csr_Ax(g.row_ptr, g.col, x64), rtol=1e-5)


@pytest.mark.parametrize("engine", ["own", "cusparse"])
def test_csr_baselines_with_hub_rows(engine):
    """Both uncompressed baselines (the hand-written CSR kernel, with hub rows
    summed by a whole CTA, and cuSPARSE) against the oracle on a graph with
    hub rows and hub columns of thousands of entries, k in {1, 8, 33}."""
    g = hub_graph()
    rows = [np.unique(np.concatenate([g.col[g.row_ptr[i]:g.row_ptr[i + 1]],
                                      np.arange(0, g.n, 1, dtype=np.int32) if i in (3, 1999) else
                                      np.zeros(0, np.int32)])) for i in range(g.n)]
    cols_hub = [np.unique(np.append(r, 17)).astype(np.int32) for r in rows]  # column 17 holds every row
    rp = np.zeros(g.n + 1, np.int64)
    rp[1:] = np.cumsum([len(r) for r in cols_hub])
    ci = np.concatenate(cols_hub)
    cg = bvg.bvg_csr_upload(rp, ci)
    xa = bvg.bvg_csr_spmv_xA if engine == "own" else bvg.bvg_csr_cusparse_xA
    ax = bvg.bvg_csr_spmv_Ax if engine == "own" else bvg.bvg_csr_cusparse_Ax
    for k in (1, 8, 33):
        x = synth.rhs(g.n, k, 40 + k)
        x64 = x.astype(np.float64)
        xt = torch.from_numpy(x).cuda()
        y = torch.full_like(xt, float("nan"))
        xa(cg, xt, y)
        np.testing.assert_allclose(y.cpu().numpy(), oracle.csr_xA(rp, ci, x64), rtol=1e-5)
        y.fill_(float("nan"))
        ax(cg, xt, y)
        np.testing.assert_allclose(y.cpu().numpy(), oracle.csr_Ax(rp, ci, x64), rtol=1e-5)


@pytest.mark.parametrize("pinned", [False, True])
@pytest.mark.parametrize("k", [1, 3, 32])
def test_host_buffer_product(pinned, k):
    """x A from host buffers, page-locked or pageable (both staged through
    device scratch): the device product bit for bit."""
    g, hg, dg, ref = graph("ragged_1037")
    x = synth.rhs(g.n, k, 17)
    xt, yt = torch.from_numpy(x), torch.zeros(g.n, k)
    if pinned:
        xt, yt = xt.pin_memory(), yt.pin_memory()
    bvg.bvg_spmv_xA_host(dg, xt, yt)
    x64 = x.astype(np.float64)
    check_close(yt.numpy(), oracle.csr_xA(g.row_ptr, g.col, x64),
                oracle.bv_xA(g.row_ptr, g.col, ref, x64, absval=True), f"host xA pinned={pinned} k={k}")
    yd = torch.empty(g.n, k, device="cuda")
    bvg.bvg_spmv_xA(dg, xt.cuda(), yd)
    assert torch.equal(yd.cpu(), yt)


def test_empty_graph():
    g = synth.Graph(50, np.zeros(51, np.int64), np.zeros(0, np.int32))
    hg, dg, ref = encode(g)
    x = torch.ones(50, 2, device="cuda")
    y = torch.full_like(x, 7.0)
    bvg.bvg_spmv_xA(dg, x, y)
    assert (y == 0).all()
    bvg.bvg_spmv_Ax(dg, x, y)
    assert (y == 0).all()
    p, it, res, rc = bvg.bvg_pagerank(dg, tol=1e-12, max_iter=50)
    np.testing.assert_allclose(p.cpu().numpy(), 1.0 / 50, rtol=1e-6)


def test_invalid_arguments():
    g, hg, dg, ref = graph("tiny_web")
    x = torch.ones(g.n, device="cuda")
    with pytest.raises(bvg.BvgError) as e:
        bvg.bvg_spmv_xA(dg, x, x)
    assert e.value.status == bvg.BVG_ERR_INVALID_ARG
    lib = bvg.load()
    hx = np.ones(g.n, np.float32)
    rc = lib.bvg_spmv_xA(dg.ptr, hx.ctypes.data, x.data_ptr(), 1, 1, None)
    assert rc == bvg.BVG_ERR_INVALID_ARG  # host pointer given to a device call
    with pytest.raises(bvg.BvgError) as e:
        bvg.bvg_pagerank(dg, k=3, p0=torch.ones(g.n, 3, device="cuda") / g.n)
    assert e.value.status == bvg.BVG_ERR_UNSUPPORTED


# ---------------------------------------------------------------- PageRank
def l1(a, b):
    return float(np.abs(np.asarray(a, np.float64).reshape(-1) - np.asarray(b, np.float64).reshape(-1)).sum())


@pytest.mark.parametrize("name", ["tiny_web", "ragged_1037", "social_20k"])
def test_pagerank_fixed_iterations(name):
    g, hg, dg, ref = graph(name)
    p, it, res, rc = bvg.bvg_pagerank(dg, tol=0.0, max_iter=20)
    want, it_o, res_o = oracle.pagerank(g.row_ptr, g.col, alpha=0.15, tol=0.0, max_iter=20)
    assert it == 20 and rc == bvg.BVG_ERR_NOT_CONVERGED
    assert l1(p.cpu().numpy(), want) <= 1e-6
    assert abs(res[0] - res_o[0]) <= 1e-6


@pytest.mark.parametrize("dangling", [0, 1])
def test_pagerank_converges_to_oracle(dangling):
    g, hg, dg, ref = graph("tiny_web")
    p, it, res, rc = bvg.bvg_pagerank(dg, tol=1e-8, max_iter=500, dangling=dangling)
    assert rc == bvg.BVG_OK and res[0] < 1e-8, (rc, it, res)
    pstar, _, _ = oracle.pagerank(g.row_ptr, g.col, alpha=0.15, tol=1e-13, max_iter=2000, dangling=dangling)
    assert l1(p.cpu().numpy(), pstar) <= 1e-6
    assert abs(float(p.double().sum()) - 1.0) < 1e-5


@pytest.mark.parametrize("k", [2, 8, 32])
def test_personalized_batch(k):
    g, hg, dg, ref = graph("tiny_web")
    seeds = synth.nodes(k, g.n, 31 + k)
    P0 = np.zeros((g.n, k), np.float32)
    P0[seeds, np.arange(k)] = 1.0
    p0 = torch.from_numpy(P0).cuda()
    p, it, res, rc = bvg.bvg_pagerank(dg, p0=p0, tol=1e-8, max_iter=500)
    assert rc == bvg.BVG_OK and (res < 1e-8).all(), (rc, it, res)
    want, _, _ = oracle.pagerank(g.row_ptr, g.col, alpha=0.15, p0=P0.astype(np.float64), tol=1e-13, max_iter=2000)
    got = p.cpu().numpy()
    for c in range(k):
        assert l1(got[:, c], want[:, c]) <= 1e-6, c
    # batched == one solve per column
    for c in (0, k - 1):
        pc, _, _, _ = bvg.bvg_pagerank(dg, p0=p0[:, c:c + 1].contiguous(), tol=1e-8, max_iter=500)
        assert l1(pc.cpu().numpy()[:, 0], got[:, c]) <= 2e-7


def test_pagerank_warm_start_and_not_converged():
    g, hg, dg, ref = graph("tiny_web")
    pstar, _, _ = oracle.pagerank(g.row_ptr, g.col, alpha=0.15, tol=1e-13, max_iter=2000)
    start = torch.from_numpy(pstar[:, 0].astype(np.float32)).cuda()
    p, it, res, rc = bvg.bvg_pagerank(dg, p_init=start, tol=1e-8, max_iter=500)
    p_u, it_u, _, _ = bvg.bvg_pagerank(dg, tol=1e-8, max_iter=500)
    assert rc == bvg.BVG_OK and it < it_u, (rc, it, it_u, res)
    assert l1(p.cpu().numpy(), pstar) <= 1e-6
    p, it, res, rc = bvg.bvg_pagerank(dg, tol=1e-12, max_iter=3)
    assert rc == bvg.BVG_ERR_NOT_CONVERGED and it == 3
    want, _, _ = oracle.pagerank(g.row_ptr, g.col, alpha=0.15, tol=0.0, max_iter=3)
    assert l1(p.cpu().numpy(), want) <= 1e-6


def test_pagerank_after_scratch_growth():
    """A wider product between two PageRank runs reallocates the pushed-weight
    scratch; the second run must not replay updates captured with the old
    buffer, and gives the same (deterministic) vector."""
    g, hg, _, _ = graph("tiny_web")
    dg = bvg.bvg_upload(hg)
    p1, it1, _, rc1 = bvg.bvg_pagerank(dg, tol=1e-8, max_iter=500)
    p1 = p1.clone()
    x = torch.rand(g.n, 4, device="cuda")
    y = torch.empty_like(x)
    bvg.bvg_spmv_xA(dg, x, y)  # k = 4 grows the scratch
    p2, it2, _, rc2 = bvg.bvg_pagerank(dg, tol=1e-8, max_iter=500)
    assert rc1 == rc2 == bvg.BVG_OK and it1 == it2
    assert torch.equal(p1, p2)


def test_pagerank_nan_reported():
    g, hg, dg, ref = graph("tiny_web")
    start = torch.full((g.n,), 1.0 / g.n, device="cuda")
    start[5] = float("nan")
    with pytest.raises(bvg.BvgError) as e:
        bvg.bvg_pagerank(dg, p_init=start, tol=1e-8, max_iter=50)
    assert e.value.status == bvg.BVG_ERR_NUMERIC


# ---------------------------------------------------------------- full size
@pytest.fixture(scope="module")
def web862k():
    g = synth.copying_model(synth.web_862k())
    hg = bvg.bvg_encode(g.row_ptr, g.col)
    ref, _ = bvg.bvg_get_refs(hg)
    return g, hg, bvg.bvg_upload(hg), ref


def test_full_size_products(web862k):
    """n = 862,664, ~19.2 M edges: every entry against the oracle."""
    g, hg, dg, ref = web862k
    x = synth.rhs(g.n, 1, synth.seed_for(2, 1))
    x64 = x.astype(np.float64)
    xt = torch.from_numpy(x).cuda()
    y = torch.empty_like(xt)
    bvg.bvg_spmv_xA(dg, xt, y)
    check_close(y.cpu().numpy(), oracle.csr_xA(g.row_ptr, g.col, x64),
                oracle.bv_xA(g.row_ptr, g.col, ref, x64, absval=True), "xA 862k")
    bvg.bvg_spmv_Ax(dg, xt, y)
    check_close(y.cpu().numpy(), oracle.csr_Ax(g.row_ptr, g.col, x64),
                oracle.bv_Ax(g.row_ptr, g.col, ref, x64, absval=True), "Ax 862k")


def test_full_size_products_wide_block(web862k):
    """n = 862,664 with k = 32 (the point-column gather): every entry of x A
    and A x^T against the oracle."""
    g, hg, dg, ref = web862k
    x = synth.rhs(g.n, 32, synth.seed_for(2, 32))
    x64 = x.astype(np.float64)
    xt = torch.from_numpy(x).cuda()
    y = torch.empty_like(xt)
    bvg.bvg_spmv_xA(dg, xt, y)
    check_close(y.cpu().numpy(), oracle.csr_xA(g.row_ptr, g.col, x64),
                oracle.bv_xA(g.row_ptr, g.col, ref, x64, absval=True), "xA 862k k=32")
    bvg.bvg_spmv_Ax(dg, xt, y)
    check_close(y.cpu().numpy(), oracle.csr_Ax(g.row_ptr, g.col, x64),
                oracle.bv_Ax(g.row_ptr, g.col, ref, x64, absval=True), "Ax 862k k=32")


def test_full_size_pagerank(web862k):
    g, hg, dg, ref = web862k
    p, it, res, rc = bvg.bvg_pagerank(dg, tol=1e-8, max_iter=1000)
    assert rc == bvg.BVG_OK and res[0] < 1e-8, (rc, it, res)
    pstar, it_o, _ = oracle.pagerank(g.row_ptr, g.col, alpha=0.15, tol=1e-12, max_iter=2000)
    assert l1(p.cpu().numpy(), pstar) <= 1e-6


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("prefix,min_len,item", [(0, 4, 8), (1, 4, 8), (-1, 32, 4), (-1, 32, 16), (-1, 1 << 20, 8)])
def test_pull_item_and_prefix_settings(name, prefix, min_len, item):
    """The pull's work items of 4, 8 or 16 entries, intervals kept whole from
    length 4 (summed from the device prefix of x, or member by member), from
    32, or never: every setting matches the oracle."""
    g, hg, dg, ref = graph(name)
    old = bvg.bvg_get_config(dg)
    bvg.bvg_set_config(dg, pull_prefix=prefix, prefix_min_len=min_len, pull_item=item)
    try:
        for k in (1, 8, 33):
            x = synth.rhs(g.n, k, synth.seed_for(1, 300 + k))
            x64 = x.astype(np.float64)
            xt = torch.from_numpy(x).cuda()
            y = torch.full_like(xt, float("nan"))
            bvg.bvg_spmv_Ax(dg, xt, y)
            check_close(y.cpu().numpy(), oracle.csr_Ax(g.row_ptr, g.col, x64),
                        oracle.bv_Ax(g.row_ptr, g.col, ref, x64, absval=True),
                        f"Ax prefix={prefix} min_len={min_len} item={item} {name} k={k}")
    finally:
        bvg.bvg_set_config(dg, **old)


def test_launch_config_variants_same_results():
    g, hg, dg, ref = graph("tiny_web")
    xt = torch.from_numpy(synth.rhs(g.n, 2, 77)).cuda()
    base_xa, base_ax = torch.empty_like(xt), torch.empty_like(xt)
    bvg.bvg_spmv_xA(dg, xt, base_xa)
    bvg.bvg_spmv_Ax(dg, xt, base_ax)
    old = bvg.bvg_get_config(dg)
    try:
        for cfg in ({"gather_pdl": 0}, {"pull_tile": 128}, {"pull_tile": 1024}):
            bvg.bvg_set_config(dg, **cfg)
            y = torch.empty_like(xt)
            bvg.bvg_spmv_xA(dg, xt, y)
            assert torch.equal(y, base_xa), cfg  # the push result does not depend on these settings
            bvg.bvg_spmv_Ax(dg, xt, y)
            assert torch.equal(y, base_ax), cfg
            bvg.bvg_set_config(dg, **old)
    finally:
        bvg.bvg_set_config(dg, **old)
    with pytest.raises(bvg.BvgError):
        bvg.bvg_set_config(dg, pull_tile=100)
    with pytest.raises(bvg.BvgError):
        bvg.bvg_set_config(dg, pull_item=5)


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("points", [0, 1])
def test_push_event_and_point_columns(name, points):
    """The push gather over the event columns (intervals as start / end events
    and a running sum) and over the point columns (every interval member its
    own entry), forced for every column block width: both match the oracle,
    and dyadic inputs match it bit for bit."""
    g, hg, dg, ref = graph(name)
    old = bvg.bvg_get_config(dg)
    bvg.bvg_set_config(dg, push_points=points, push_fused=0)
    try:
        for k in (1, 2, 8, 33):
            x = synth.rhs(g.n, k, synth.seed_for(1, 400 + k))
            x64 = x.astype(np.float64)
            xt = torch.from_numpy(x).cuda()
            y = torch.full_like(xt, float("nan"))
            bvg.bvg_spmv_xA(dg, xt, y)
            check_close(y.cpu().numpy(), oracle.csr_xA(g.row_ptr, g.col, x64),
                        oracle.bv_xA(g.row_ptr, g.col, ref, x64, absval=True), f"xA points={points} {name} k={k}")
        for k in (1, 4, 32):
            x = synth.dyadic_rhs(g.n, k, synth.seed_for(1, 500 + k))
            xt = torch.from_numpy(x).cuda()
            y = torch.empty_like(xt)
            bvg.bvg_spmv_xA(dg, xt, y)
            np.testing.assert_array_equal(y.cpu().numpy().astype(np.float64), oracle.csr_xA(g.row_ptr, g.col, x))
    finally:
        bvg.bvg_set_config(dg, **old)
    info = bvg.bvg_dev_layout(dg)
    if points:
        assert info["point_entries"] == bvg.bvg_stats(hg)["nnz_diff"]


@pytest.mark.parametrize("points", [0, 1])
def test_pagerank_event_and_point_columns(points):
    """PageRank (one vector and eight personalized ones) with the gather forced
    onto either column layout: both converge to the oracle's vectors."""
    g, hg, dg, ref = graph("social_20k")
    old = bvg.bvg_get_config(dg)
    bvg.bvg_set_config(dg, push_points=points, push_fused=0)
    try:
        p, it, res, rc = bvg.bvg_pagerank(dg, tol=1e-8, max_iter=1000)
        assert rc == bvg.BVG_OK and res[0] < 1e-8, (rc, it, res)
        pstar, _, _ = oracle.pagerank(g.row_ptr, g.col, alpha=0.15, tol=1e-13, max_iter=2000)
        assert l1(p.cpu().numpy(), pstar) <= 1e-6
        k = 8
        P0 = np.zeros((g.n, k), np.float32)
        P0[synth.nodes(k, g.n, 77), np.arange(k)] = 1.0
        p, it, res, rc = bvg.bvg_pagerank(dg, p0=torch.from_numpy(P0).cuda(), tol=1e-8, max_iter=1000)
        assert rc == bvg.BVG_OK and (res < 1e-8).all(), (rc, it, res)
        want, _, _ = oracle.pagerank(g.row_ptr, g.col, alpha=0.15, p0=P0.astype(np.float64), tol=1e-13,
                                     max_iter=2000)
        got = p.cpu().numpy()
        for c in range(k):
            assert l1(got[:, c], want[:, c]) <= 1e-6, c
    finally:
        bvg.bvg_set_config(dg, **old)


def hub_graph():
    """A web-like graph with hub rows: a few rows hold every other id (1,500
    single entries, no runs: about a hundred work items or more), some of
    them adjacent so that they reference one another and fall in the halo of
    the next row tile."""
    g = synth.copying_model(synth.GraphSpec(n=3000, seed=9, p_copy=0.7, fidelity=0.97, extra_mean=0.8,
                                            fresh_mean=6.0, q_run=0.25, gap_mean=30.0))
    even, odd = {0, 700, 2048, 2999}, {1, 63, 65, 1500, 2047}
    rows = [np.arange(i % 2, g.n, 2, dtype=np.int32) if i in even | odd else g.col[g.row_ptr[i]:g.row_ptr[i + 1]]
            for i in range(g.n)]
    rp = np.zeros(g.n + 1, np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    return synth.Graph(g.n, rp, np.concatenate(rows).astype(np.int32))


@pytest.mark.parametrize("tile,item", [(64, 4), (512, 8), (2048, 16)])
def test_pull_hub_rows(tile, item):
    """Rows with more than 32 work items are summed by the whole row tile:
    results match the oracle for every column block, dyadic inputs bit for
    bit, and repeated products are identical."""
    g = hub_graph()
    hg, dg, ref = encode(g)
    bvg.bvg_set_config(dg, pull_tile=tile, pull_item=item)
    for k in (1, 2, 8, 33):
        x = synth.rhs(g.n, k, synth.seed_for(1, 800 + k))
        x64 = x.astype(np.float64)
        xt = torch.from_numpy(x).cuda()
        y = torch.full_like(xt, float("nan"))
        bvg.bvg_spmv_Ax(dg, xt, y)
        check_close(y.cpu().numpy(), oracle.csr_Ax(g.row_ptr, g.col, x64),
                    oracle.bv_Ax(g.row_ptr, g.col, ref, x64, absval=True), f"Ax hubs tile={tile} item={item} k={k}")
        y2 = torch.empty_like(xt)
        bvg.bvg_spmv_Ax(dg, xt, y2)
        assert torch.equal(y, y2)
    for k in (1, 32):
        x = synth.dyadic_rhs(g.n, k, synth.seed_for(1, 900 + k))
        xt = torch.from_numpy(x).cuda()
        y = torch.empty_like(xt)
        bvg.bvg_spmv_Ax(dg, xt, y)
        np.testing.assert_array_equal(y.cpu().numpy().astype(np.float64), oracle.csr_Ax(g.row_ptr, g.col, x))


def hub_column_graph():
    """A web-like graph with two hub columns: every row links to node 5 with
    probability 1/2 and to node 2500 with probability 3/10, independently, so
    the reference copies cannot absorb them: columns 5 and 2500 of A' hold
    about 1,300 and 1,000 entries."""
    g = synth.copying_model(synth.GraphSpec(n=3000, seed=11, p_copy=0.7, fidelity=0.97, extra_mean=0.8,
                                            fresh_mean=6.0, q_run=0.25, gap_mean=30.0))
    u = synth.uniform(2 * g.n, synth.seed_for(1, 77)).reshape(2, g.n)
    rows = []
    for i in range(g.n):
        r = set(g.col[g.row_ptr[i]:g.row_ptr[i + 1]].tolist())
        if u[0, i] < 0.5:
            r.add(5)
        if u[1, i] < 0.3:
            r.add(2500)
        rows.append(np.array(sorted(r), np.int32))
    rp = np.zeros(g.n + 1, np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    return synth.Graph(g.n, rp, np.concatenate(rows))


@pytest.mark.parametrize("points", [-1, 1])
def test_push_hub_columns(points):
    """Columns with more than 256 tail entries are summed by the whole CTA
    (wide column blocks over point columns): x A matches the oracle for every
    column block, dyadic inputs bit for bit, repeated products are identical,
    and 8 personalized PageRank vectors converge to the oracle's."""
    g = hub_column_graph()
    hg, dg, ref = encode(g)
    cnt = np.diff(bvg.bvg_point_cols(hg)["colp"].astype(np.int64))
    assert cnt[5] > 4 + 256 and cnt[2500] > 4 + 256
    bvg.bvg_set_config(dg, push_points=points)
    for k in (1, 2, 8, 16, 32, 33):
        x = synth.rhs(g.n, k, synth.seed_for(1, 1000 + k))
        x64 = x.astype(np.float64)
        xt = torch.from_numpy(x).cuda()
        y = torch.full_like(xt, float("nan"))
        bvg.bvg_spmv_xA(dg, xt, y)
        check_close(y.cpu().numpy(), oracle.csr_xA(g.row_ptr, g.col, x64),
                    oracle.bv_xA(g.row_ptr, g.col, ref, x64, absval=True), f"xA hub columns points={points} k={k}")
        y2 = torch.empty_like(xt)
        bvg.bvg_spmv_xA(dg, xt, y2)
        assert torch.equal(y, y2)
    for k in (8, 32):
        x = synth.dyadic_rhs(g.n, k, synth.seed_for(1, 1100 + k))
        xt = torch.from_numpy(x).cuda()
        y = torch.empty_like(xt)
        bvg.bvg_spmv_xA(dg, xt, y)
        np.testing.assert_array_equal(y.cpu().numpy().astype(np.float64), oracle.csr_xA(g.row_ptr, g.col, x))
    k = 8
    P0 = np.zeros((g.n, k), np.float32)
    P0[synth.nodes(k, g.n, 78), np.arange(k)] = 1.0
    p, it, res, rc = bvg.bvg_pagerank(dg, p0=torch.from_numpy(P0).cuda(), tol=1e-8, max_iter=1000)
    assert rc == bvg.BVG_OK and (res < 1e-8).all(), (rc, it, res)
    want, _, _ = oracle.pagerank(g.row_ptr, g.col, alpha=0.15, p0=P0.astype(np.float64), tol=1e-13, max_iter=2000)
    for c in range(k):
        assert l1(p.cpu().numpy()[:, c], want[:, c]) <= 1e-6, c


@pytest.mark.parametrize("window,max_chain", [(1, 1), (3, 2), (5, 3), (7, 1), (10, 3), (15, 2), (31, 1)])
def test_other_windows_and_chain_bounds(window, max_chain):
    """Encodings with a shorter reference window W (Sec. 4) or chain bound R:
    both products and PageRank match the oracle (the oracle decodes its own
    references from the same encoding)."""
    g = synth.copying_model(synth.tiny_web())
    hg = bvg.bvg_encode(g.row_ptr, g.col, window=window, max_chain=max_chain)
    ref, depth = bvg.bvg_get_refs(hg)
    assert depth.max() <= max_chain and np.all((ref < 0) | (np.arange(g.n) - ref <= window))
    dg = bvg.bvg_upload(hg)
    for k in (1, 8, 33):
        x = synth.rhs(g.n, k, synth.seed_for(1, 1200 + k))
        x64 = x.astype(np.float64)
        xt = torch.from_numpy(x).cuda()
        y = torch.full_like(xt, float("nan"))
        bvg.bvg_spmv_xA(dg, xt, y)
        check_close(y.cpu().numpy(), oracle.csr_xA(g.row_ptr, g.col, x64),
                    oracle.bv_xA(g.row_ptr, g.col, ref, x64, absval=True), f"xA W={window} R={max_chain} k={k}")
        y.fill_(float("nan"))
        bvg.bvg_spmv_Ax(dg, xt, y)
        check_close(y.cpu().numpy(), oracle.csr_Ax(g.row_ptr, g.col, x64),
                    oracle.bv_Ax(g.row_ptr, g.col, ref, x64, absval=True), f"Ax W={window} R={max_chain} k={k}")
    p, it, res, rc = bvg.bvg_pagerank(dg, tol=1e-8, max_iter=1000)
    assert rc == bvg.BVG_OK and res[0] < 1e-8
    pstar, _, _ = oracle.pagerank(g.row_ptr, g.col, alpha=0.15, tol=1e-13, max_iter=2000)
    assert l1(p.cpu().numpy(), pstar) <= 1e-6


@pytest.mark.parametrize("after", [0, 3, 9])
def test_upload_allocation_failure(after):
    """A device allocation of bvg_upload that fails (the allocation-failure
    hook makes the given checkpoint fail) returns BVG_ERR_OOM and releases
    what was allocated; the next upload of the same graph works and gives the
    oracle's product."""
    g, hg, _, ref = graph("tiny_web")
    free0, _ = torch.cuda.mem_get_info()
    bvg.bvg_debug_fail_alloc(after)
    try:
        with pytest.raises(bvg.BvgError) as e:
            bvg.bvg_upload(hg)
        assert e.value.status == bvg.BVG_ERR_OOM
    finally:
        bvg.bvg_debug_fail_alloc(-1)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free0 - free1 < 8 << 20  # nothing of the failed upload is kept (allocator granularity aside)
    dg = bvg.bvg_upload(hg)
    x = synth.rhs(g.n, 1, 5)
    xt = torch.from_numpy(x).cuda()
    y = torch.empty_like(xt)
    bvg.bvg_spmv_xA(dg, xt, y)
    x64 = x.astype(np.float64)
    check_close(y.cpu().numpy(), oracle.csr_xA(g.row_ptr, g.col, x64),
                oracle.bv_xA(g.row_ptr, g.col, ref, x64, absval=True), "xA after a failed upload")

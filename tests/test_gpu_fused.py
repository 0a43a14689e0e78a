"""The fused one-vector x A kernel (one launch: chain weights and the column
gather of Proposition 1's left product in shared memory, exact fixed-point
sums) through the C ABI against the CPU oracle.

Exactness pin: on tiles whose inputs span few binades every sum is exact, so
y_j is the exact x A rounded once to FP32. The oracle's FP64 sum is within
about 1e-16 (relative) of the exact value, so its rounding to FP32 must equal
the kernel's result except when the FP64 sum sits within that distance of a
rounding boundary between two floats (rare); the test demands equality on at
least 99.9 % of the columns and at most one unit in the last place anywhere.
Everywhere: the per-entry tolerance of the other parity tests.
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


def check_close(got, want, mag, what):
    err = np.abs(got.astype(np.float64) - want)
    bound = RTOL * np.maximum(np.abs(want), mag) + 1e-300
    bad = np.nonzero(~(err <= bound))
    assert bad[0].size == 0, f"{what}: {bad[0].size} entries off, worst {err.max():.3e} at {np.argmax(err)}"


def ulps(a32, b32):
    """Distance in units in the last place between two FP32 arrays of one sign."""
    ia = a32.astype(np.float32).view(np.int32).astype(np.int64)
    ib = b32.astype(np.float32).view(np.int32).astype(np.int64)
    return np.abs(ia - ib)


GRAPHS = {
    "tiny_web": lambda: synth.copying_model(synth.tiny_web()),
    "ragged_1037": lambda: synth.copying_model(synth.replace(synth.tiny_web(), n=1037, seed=77)),
    "web_50k": lambda: synth.copying_model(synth.web_small(50_000, synth.seed_for(8, 1))),
    "long_runs": lambda: synth.copying_model(synth.GraphSpec(n=5000, seed=6, p_copy=0.6, fidelity=0.95,
                                                             extra_mean=1.0, fresh_mean=300, q_run=0.9,
                                                             run_min=100, run_max=900, gap_mean=50.0)),
    "social_20k": lambda: synth.copying_model(synth.replace(synth.social_5m4(), n=20_000)),
}
_cache = {}


def graph(name):
    if name not in _cache:
        g = GRAPHS[name]()
        hg = bvg.bvg_encode(g.row_ptr, g.col)
        ref, _ = bvg.bvg_get_refs(hg)
        dg = bvg.bvg_upload(hg)
        bvg.bvg_set_config(dg, push_fused=1)  # forced, also where rows outside the window are common
        _cache[name] = (g, hg, dg, ref)
    return _cache[name]


def run_xA(dg, x):
    xt = torch.from_numpy(x).cuda()
    y = torch.full_like(xt, float("nan"))
    bvg.bvg_spmv_xA(dg, xt, y)
    bvg.bvg_device_check(dg)
    return y.cpu().numpy()


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("kind", ["uniform", "signed", "wide"])
def test_fused_matches_oracle(name, kind):
    g, hg, dg, ref = graph(name)
    x = synth.input_kind(kind, g.n, 1, synth.seed_for(8, 10 + len(kind)))
    x64 = x.astype(np.float64)
    got = run_xA(dg, x)
    check_close(got, oracle.csr_xA(g.row_ptr, g.col, x64), oracle.bv_xA(g.row_ptr, g.col, ref, x64, absval=True),
                f"fused {kind} {name}")


@pytest.mark.parametrize("name", ["tiny_web", "ragged_1037", "web_50k"])
def test_fused_is_the_exact_sum_rounded_once(name):
    """x ~ U[2^-10, 1) on graphs with locality (every tile within the exact
    path's range and reading no row outside its window): y_j is the exact sum
    rounded once to FP32."""
    g, hg, dg, ref = graph(name)
    x = (np.float64(2.0 ** -10) + (1 - 2.0 ** -10) * synth.uniform(g.n, synth.seed_for(8, 40))).astype(np.float32)
    got = run_xA(dg, x.reshape(-1, 1))[:, 0]
    want = oracle.csr_xA(g.row_ptr, g.col, x.astype(np.float64).reshape(-1, 1))[:, 0]
    want32 = want.astype(np.float32)
    d = ulps(got, want32)
    assert d.max() <= 1, d.max()
    assert np.mean(d == 0) >= 0.999, np.mean(d == 0)


def test_fused_signed_dyadic_bit_exact():
    for name in GRAPHS:
        g, hg, dg, ref = graph(name)
        x = synth.signed_dyadic_rhs(g.n, 1, synth.seed_for(8, 50))
        np.testing.assert_array_equal(run_xA(dg, x).astype(np.float64), oracle.csr_xA(g.row_ptr, g.col, x))


def test_fused_equals_other_layouts_within_tolerance_and_is_deterministic():
    g, hg, dg, ref = graph("web_50k")
    x = synth.rhs(g.n, 1, synth.seed_for(8, 60))
    y1 = run_xA(dg, x)
    y2 = run_xA(dg, x)
    np.testing.assert_array_equal(y1, y2)
    bvg.bvg_set_config(dg, push_fused=0)
    try:
        y3 = run_xA(dg, x)
    finally:
        bvg.bvg_set_config(dg, push_fused=1)
    x64 = x.astype(np.float64)
    check_close(y3, y1.astype(np.float64), oracle.bv_xA(g.row_ptr, g.col, ref, x64, absval=True), "fused vs two-kernel")


def test_fused_nonfinite_inputs():
    """A NaN and an infinity in x: the tiles that read them take the
    compensated path, so exactly the columns that the compressed formula
    (the oracle's own compressed product, Sec. 4) makes non-finite are
    non-finite -- a superset of the plain product's, since a non-finite z_k
    times +1 and -1 along a reference chain does not cancel -- and every other
    column matches the oracle."""
    g, hg, dg, ref = graph("web_50k")
    x = synth.rhs(g.n, 1, synth.seed_for(8, 70))
    x[1234, 0] = np.nan
    x[40000, 0] = np.inf
    got = run_xA(dg, x)
    x64 = x.astype(np.float64)
    want = oracle.csr_xA(g.row_ptr, g.col, x64)
    bad = ~np.isfinite(oracle.bv_xA(g.row_ptr, g.col, ref, x64))
    assert bad.any() and np.all(bad[~np.isfinite(want)])
    np.testing.assert_array_equal(~np.isfinite(got), bad)
    mag = oracle.bv_xA(g.row_ptr, g.col, ref, np.where(np.isfinite(x64), x64, 0.0), absval=True)
    check_close(got[~bad], want[~bad], mag[~bad], "finite columns")


def test_fused_rows_outside_the_window():
    """A graph whose rows link far away (every row also links to row
    (7919 i) mod n): the tiles read rows outside their window, whose chain
    weights come from global memory; the default keeps such a graph on the
    two-kernel product, the forced fused kernel matches the oracle too."""
    base = synth.copying_model(synth.web_small(30_000, synth.seed_for(8, 80)))
    rows = []
    for i in range(base.n):
        r = set(base.col[base.row_ptr[i]:base.row_ptr[i + 1]].tolist())
        r.add((7919 * i) % base.n)
        rows.append(np.array(sorted(r), np.int32))
    rp = np.zeros(base.n + 1, np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    g = synth.Graph(base.n, rp, np.concatenate(rows))
    hg = bvg.bvg_encode(g.row_ptr, g.col)
    ref, _ = bvg.bvg_get_refs(hg)
    dg = bvg.bvg_upload(hg)
    for fused in (-1, 1):
        bvg.bvg_set_config(dg, push_fused=fused)
        for kind in ("uniform", "wide"):
            x = synth.input_kind(kind, g.n, 1, synth.seed_for(8, 90))
            x64 = x.astype(np.float64)
            check_close(run_xA(dg, x), oracle.csr_xA(g.row_ptr, g.col, x64),
                        oracle.bv_xA(g.row_ptr, g.col, ref, x64, absval=True), f"far rows fused={fused} {kind}")


@pytest.mark.parametrize("dangling", [0, 1])
def test_fused_pagerank(dangling):
    """PageRank with one fused kernel per update: converges to the oracle's
    fixed point; a personalised teleport vector too."""
    g, hg, dg, ref = graph("web_50k")
    p, it, res, rc = bvg.bvg_pagerank(dg, tol=1e-8, max_iter=1000, dangling=dangling)
    assert rc == bvg.BVG_OK and res[0] < 1e-8, (rc, it, res)
    pstar, _, _ = oracle.pagerank(g.row_ptr, g.col, alpha=0.15, tol=1e-13, max_iter=3000, dangling=dangling)
    assert float(np.abs(p.cpu().numpy().astype(np.float64) - pstar[:, 0]).sum()) <= 1e-6
    p0 = np.zeros((g.n, 1), np.float32)
    p0[synth.nodes(1, g.n, 5), 0] = 1.0
    p, it, res, rc = bvg.bvg_pagerank(dg, p0=torch.from_numpy(p0).cuda(), tol=1e-8, max_iter=1000,
                                      dangling=dangling)
    assert rc == bvg.BVG_OK, (rc, it, res)
    want, _, _ = oracle.pagerank(g.row_ptr, g.col, alpha=0.15, p0=p0.astype(np.float64), tol=1e-13, max_iter=3000,
                                 dangling=dangling)
    assert float(np.abs(p.cpu().numpy().reshape(-1).astype(np.float64) - want[:, 0]).sum()) <= 1e-6
    bvg.bvg_device_check(dg)


def test_fused_pagerank_fixed_iterations_match_two_kernel_updates():
    """20 updates with the fused kernel and with the two-kernel update: both
    the oracle's 20th iterate within 1e-6 in L1."""
    g, hg, dg, ref = graph("tiny_web")
    want, _, _ = oracle.pagerank(g.row_ptr, g.col, alpha=0.15, tol=0.0, max_iter=20)
    for fused in (1, 0):
        bvg.bvg_set_config(dg, push_fused=fused)
        p, it, res, rc = bvg.bvg_pagerank(dg, tol=0.0, max_iter=20)
        assert it == 20
        assert float(np.abs(p.cpu().numpy().astype(np.float64) - want[:, 0]).sum()) <= 1e-6, fused
    bvg.bvg_set_config(dg, push_fused=1)


def test_fused_full_size(web862k_fused):
    """n = 862,664 (the bench's workload and launch): every entry against the
    oracle, uniform and wide-range x, and the default uses the fused kernel."""
    g, hg, dg, ref = web862k_fused
    assert bvg.bvg_get_config(dg)["push_fused"] == -1
    L = bvg.bvg_dev_layout(dg)
    for kind in ("uniform", "wide"):
        x = synth.input_kind(kind, g.n, 1, synth.seed_for(2, 1) if kind == "uniform" else synth.seed_for(8, 99))
        x64 = x.astype(np.float64)
        check_close(run_xA(dg, x), oracle.csr_xA(g.row_ptr, g.col, x64),
                    oracle.bv_xA(g.row_ptr, g.col, ref, x64, absval=True), f"862k fused {kind}")
    bvg.bvg_trace_enable(dg, True)
    bvg.bvg_trace_read(dg)
    run_xA(dg, synth.rhs(g.n, 1, 3))
    tr = bvg.bvg_trace_read(dg)
    bvg.bvg_trace_enable(dg, False)
    assert set(tr) == {"push_fused"}, tr
    assert L["n"] == g.n


@pytest.fixture(scope="module")
def web862k_fused():
    g = synth.copying_model(synth.web_862k())
    hg = bvg.bvg_encode(g.row_ptr, g.col)
    ref, _ = bvg.bvg_get_refs(hg)
    return g, hg, bvg.bvg_upload(hg), ref


def transpose(g):
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    order = np.lexsort((src, g.col))
    tp = np.zeros(g.n + 1, np.int64)
    tp[1:] = np.cumsum(np.bincount(g.col, minlength=g.n))
    return tp, src[order].astype(np.int32)


@pytest.mark.parametrize("name", ["tiny_web", "ragged_1037", "web_50k"])
def test_products_through_the_transpose(name):
    """A x^T as the push on an encoding of A^T (x A^T), and x A as the pull on
    it (the paper's own PageRank choice): both against the oracle's products
    of A."""
    g = GRAPHS[name]()
    tp, tc = transpose(g)
    hgT = bvg.bvg_encode(tp, tc)
    refT, _ = bvg.bvg_get_refs(hgT)
    dgT = bvg.bvg_upload(hgT)
    for kind in ("uniform", "signed"):
        x = synth.input_kind(kind, g.n, 1, synth.seed_for(8, 120 + len(kind)))
        x64 = x.astype(np.float64)
        xt = torch.from_numpy(x).cuda()
        y = torch.empty_like(xt)
        bvg.bvg_spmv_xA(dgT, xt, y)
        check_close(y.cpu().numpy(), oracle.csr_Ax(g.row_ptr, g.col, x64),
                    oracle.bv_xA(tp, tc, refT, x64, absval=True), f"A x^T as push on A^T {kind} {name}")
        bvg.bvg_spmv_Ax(dgT, xt, y)
        check_close(y.cpu().numpy(), oracle.csr_xA(g.row_ptr, g.col, x64),
                    oracle.bv_Ax(tp, tc, refT, x64, absval=True), f"x A as pull on A^T {kind} {name}")

"""GPU parity on signed and wide-range right-hand sides, and on degenerate
graphs, through the C ABI against the CPU oracle element by element.

The product is defined for any real x (Sec. 1); signed x is where the
compensated sums along reference chains (Proposition 1), the running interval
prefix of the push gather and the pull's row sums meet cancellation. The
tolerance is the one of the other parity tests, derived from the arithmetic:
|y - y*| <= 1e-5 * max(|y*|, s) per entry, s the sum of the magnitudes of the
terms the compressed formula adds (computed by the oracle on its own
difference rows with |x|). Signed dyadic inputs (integers / 2^10) make every
partial sum exact, so there the results match bit for bit.

Input recipes: 'signed' x ~ U(-1, 1); 'wide' x = +-m 2^e, m ~ U[1, 2), e a
uniform integer in [-20, 20] (magnitudes spread over 40 binades)."""
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
    bad = np.nonzero(~(err <= bound))  # NaN (an entry never written) counts as a mismatch
    assert bad[0].size == 0, f"{what}: {bad[0].size} entries off, worst {err.max():.3e} at {np.argmax(err)}"


GRAPHS = {
    "tiny_web": lambda: synth.copying_model(synth.tiny_web()),
    "ragged_1037": lambda: synth.copying_model(synth.replace(synth.tiny_web(), n=1037, seed=77)),
    "social_20k": lambda: synth.copying_model(synth.replace(synth.social_5m4(), n=20_000)),
    "long_runs": lambda: synth.copying_model(synth.GraphSpec(n=5000, seed=6, p_copy=0.6, fidelity=0.95,
                                                             extra_mean=1.0, fresh_mean=300, q_run=0.9,
                                                             run_min=100, run_max=900, gap_mean=50.0)),
}
_cache = {}


def graph(name):
    if name not in _cache:
        g = GRAPHS[name]()
        hg = bvg.bvg_encode(g.row_ptr, g.col)
        ref, _ = bvg.bvg_get_refs(hg)
        _cache[name] = (g, hg, bvg.bvg_upload(hg), ref)
    return _cache[name]


def both_products(g, dg, ref, x, what):
    x64 = x.astype(np.float64)
    xt = torch.from_numpy(x).cuda()
    y = torch.full_like(xt, float("nan"))
    bvg.bvg_spmv_xA(dg, xt, y)
    check_close(y.cpu().numpy(), oracle.csr_xA(g.row_ptr, g.col, x64),
                oracle.bv_xA(g.row_ptr, g.col, ref, x64, absval=True), "xA " + what)
    y.fill_(float("nan"))
    bvg.bvg_spmv_Ax(dg, xt, y)
    check_close(y.cpu().numpy(), oracle.csr_Ax(g.row_ptr, g.col, x64),
                oracle.bv_Ax(g.row_ptr, g.col, ref, x64, absval=True), "Ax " + what)


@pytest.mark.parametrize("kind", ["signed", "wide"])
@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("k", [1, 2, 8, 33])
def test_signed_products_match_oracle(kind, name, k):
    g, hg, dg, ref = graph(name)
    x = synth.input_kind(kind, g.n, k, synth.seed_for(6, 10 * k + (kind == "wide")))
    both_products(g, dg, ref, x, f"{kind} {name} k={k}")


@pytest.mark.parametrize("points", [0, 1])
@pytest.mark.parametrize("name", list(GRAPHS))
def test_signed_dyadic_bit_exact_both_column_layouts(name, points):
    """Signed dyadic x: both products equal the oracle bit for bit, with the
    push gather forced onto the event columns and onto the point columns."""
    g, hg, dg, ref = graph(name)
    old = bvg.bvg_get_config(dg)
    bvg.bvg_set_config(dg, push_points=points, push_fused=0)
    try:
        for k in (1, 4, 32):
            x = synth.signed_dyadic_rhs(g.n, k, synth.seed_for(6, 100 + k))
            xt = torch.from_numpy(x).cuda()
            y = torch.empty_like(xt)
            bvg.bvg_spmv_xA(dg, xt, y)
            np.testing.assert_array_equal(y.cpu().numpy().astype(np.float64), oracle.csr_xA(g.row_ptr, g.col, x))
            bvg.bvg_spmv_Ax(dg, xt, y)
            np.testing.assert_array_equal(y.cpu().numpy().astype(np.float64), oracle.csr_Ax(g.row_ptr, g.col, x))
    finally:
        bvg.bvg_set_config(dg, **old)


@pytest.mark.parametrize("kind,layouts", [("signed", ((1, -1), (1, 0), (0, 0))), ("wide", ((1, -1), (1, 0)))])
def test_signed_push_column_layouts(kind, layouts):
    """Signed x through the fused one-vector kernel, the point-column gather
    and the event-column gather; wide-range x through the first two. (The
    event gather's running FP32 interval sum carries an error relative to the
    intervals that opened and closed earlier in its tile, not only to the
    column's own terms, so wide-range x can exceed the per-entry tolerance
    there: that layout is not the default for any column block.)"""
    g, hg, dg, ref = graph("tiny_web")
    old = bvg.bvg_get_config(dg)
    try:
        for points, fused in layouts:
            bvg.bvg_set_config(dg, push_points=points, push_fused=fused)
            for k in (1, 2, 8, 33):
                x = synth.input_kind(kind, g.n, k, synth.seed_for(6, 200 + k))
                x64 = x.astype(np.float64)
                xt = torch.from_numpy(x).cuda()
                y = torch.full_like(xt, float("nan"))
                bvg.bvg_spmv_xA(dg, xt, y)
                check_close(y.cpu().numpy(), oracle.csr_xA(g.row_ptr, g.col, x64),
                            oracle.bv_xA(g.row_ptr, g.col, ref, x64, absval=True),
                            f"xA {kind} points={points} fused={fused} k={k}")
    finally:
        bvg.bvg_set_config(dg, **old)


def test_signed_batch_matches_oracle():
    """The multi-graph batch on signed x: the one-graph product bit for bit and
    the oracle within the tolerance."""
    gs = [synth.copying_model(synth.web_small(n, synth.seed_for(6, 300 + i))) for i, n in
          enumerate((1000, 4097, 20000))]
    dgs, refs = [], []
    for g in gs:
        hg = bvg.bvg_encode(g.row_ptr, g.col)
        refs.append(bvg.bvg_get_refs(hg)[0])
        dgs.append(bvg.bvg_upload(hg))
    b = bvg.bvg_batch_create(dgs)
    for k in (1, 8):
        xs = [torch.from_numpy(synth.signed_rhs(g.n, k, synth.seed_for(6, 310 + i))).cuda() for i, g in enumerate(gs)]
        if k == 1:
            xs = [x.reshape(-1) for x in xs]
        ys = [torch.full_like(x, float("nan")) for x in xs]
        bvg.bvg_batch_spmv_xA(b, xs, ys)
        torch.cuda.synchronize()
        for g, d, ref, x, y in zip(gs, dgs, refs, xs, ys):
            y1 = torch.empty_like(x)
            bvg.bvg_spmv_xA(d, x, y1)
            assert torch.equal(y, y1)
            x64 = x.cpu().numpy().astype(np.float64).reshape(g.n, -1)
            check_close(y.cpu().numpy().reshape(g.n, -1), oracle.csr_xA(g.row_ptr, g.col, x64),
                        oracle.bv_xA(g.row_ptr, g.col, ref, x64, absval=True), f"batch signed k={k}")


def _csr(rows, n):
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate([np.asarray(r, np.int32) for r in rows]) if rp[-1] else np.zeros(0, np.int32)
    return synth.Graph(n, rp, col)


def degenerate(case):
    if case == "one_row":
        return _csr([[0]], 1)
    if case == "one_row_no_edge":
        return _csr([[]], 1)
    if case == "identical_rows":  # every row a copy of its reference: A' holds only the roots' rows
        return _csr([[3, 17, 18, 19, 20, 21, 250] for _ in range(300)], 300)
    if case == "full_interval":  # one row is a single interval over every id
        n = 700
        return _csr([list(range(n)) if i == 5 else [i] for i in range(n)], n)
    if case == "full_rows":  # every row holds every id: intervals everywhere, copies of them
        n = 600
        return _csr([list(range(n)) for _ in range(n)], n)
    if case == "self_loops":
        n = 257
        return _csr([[i] for i in range(n)], n)
    raise KeyError(case)


@pytest.mark.parametrize("case", ["one_row", "one_row_no_edge", "identical_rows", "full_interval", "full_rows",
                                  "self_loops"])
def test_degenerate_graphs_on_gpu(case):
    """Degenerate graphs through the kernels: a single row (with and without
    its self-loop), rows that all copy their reference, one row that is a
    single interval over every id, every row full, only self-loops. Both
    products for k in {1, 4, 33} with uniform and signed x, signed dyadic x
    bit for bit, and PageRank to the oracle's fixed point."""
    g = degenerate(case)
    hg = bvg.bvg_encode(g.row_ptr, g.col)
    ref, _ = bvg.bvg_get_refs(hg)
    dg = bvg.bvg_upload(hg)
    for k in (1, 4, 33):
        for kind in ("uniform", "signed"):
            x = synth.input_kind(kind, g.n, k, synth.seed_for(6, 400 + k))
            both_products(g, dg, ref, x, f"{case} {kind} k={k}")
        x = synth.signed_dyadic_rhs(g.n, k, synth.seed_for(6, 450 + k))
        xt = torch.from_numpy(x).cuda()
        y = torch.empty_like(xt)
        bvg.bvg_spmv_xA(dg, xt, y)
        np.testing.assert_array_equal(y.cpu().numpy().astype(np.float64), oracle.csr_xA(g.row_ptr, g.col, x))
        bvg.bvg_spmv_Ax(dg, xt, y)
        np.testing.assert_array_equal(y.cpu().numpy().astype(np.float64), oracle.csr_Ax(g.row_ptr, g.col, x))
    p, it, res, rc = bvg.bvg_pagerank(dg, tol=1e-9, max_iter=2000)
    assert rc == bvg.BVG_OK, (rc, it, res)
    pstar, _, _ = oracle.pagerank(g.row_ptr, g.col, alpha=0.15, tol=1e-13, max_iter=5000)
    assert float(np.abs(p.cpu().numpy().astype(np.float64) - pstar[:, 0]).sum()) <= 1e-6


@pytest.fixture(scope="module")
def web862k():
    g = synth.copying_model(synth.web_862k())
    hg = bvg.bvg_encode(g.row_ptr, g.col)
    ref, _ = bvg.bvg_get_refs(hg)
    return g, hg, bvg.bvg_upload(hg), ref


@pytest.mark.parametrize("kind", ["signed", "wide"])
def test_full_size_signed_products(web862k, kind):
    """n = 862,664, ~19.2 M edges, k = 1 (the bench's launch configuration):
    every entry of both products against the oracle on signed and wide-range x."""
    g, hg, dg, ref = web862k
    x = synth.input_kind(kind, g.n, 1, synth.seed_for(6, 500 + (kind == "wide")))
    both_products(g, dg, ref, x, f"862k {kind}")


def test_full_size_signed_dyadic_bit_exact(web862k):
    g, hg, dg, ref = web862k
    x = synth.signed_dyadic_rhs(g.n, 1, synth.seed_for(6, 510))
    xt = torch.from_numpy(x).cuda()
    y = torch.empty_like(xt)
    bvg.bvg_spmv_xA(dg, xt, y)
    np.testing.assert_array_equal(y.cpu().numpy().astype(np.float64), oracle.csr_xA(g.row_ptr, g.col, x))
    bvg.bvg_spmv_Ax(dg, xt, y)
    np.testing.assert_array_equal(y.cpu().numpy().astype(np.float64), oracle.csr_Ax(g.row_ptr, g.col, x))

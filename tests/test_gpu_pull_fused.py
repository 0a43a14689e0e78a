"""The one-vector A x^T in one launch (Sec. 4: y_i = y_{r_i} + sum_j A'_ij
x_j; each row tile's difference sums and reference chains in shared memory,
exact fixed-point sums) through the C ABI against the CPU oracle.

Exactness pin: on tiles whose x span few binades every sum is exact, so y_i
is the exact A x^T rounded once to FP32; the oracle's FP64 sum rounded to
FP32 must equal it except within about 1e-16 of a rounding boundary (rare):
equality on at least 99.9 % of the rows and at most one unit in the last
place anywhere. Everywhere: the per-entry tolerance of the other parity
tests, 1e-5 * max(|y*|, s), s the oracle's magnitudes on its own A'.
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

GRAPHS = {
    "tiny_web": lambda: synth.copying_model(synth.tiny_web()),
    "ragged_1037": lambda: synth.copying_model(synth.replace(synth.tiny_web(), n=1037, seed=77)),
    "web_50k": lambda: synth.copying_model(synth.web_small(50_000, synth.seed_for(8, 1))),
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


def check_close(got, want, mag, what):
    err = np.abs(got.astype(np.float64) - want)
    bad = np.nonzero(~(err <= RTOL * np.maximum(np.abs(want), mag) + 1e-300))
    assert bad[0].size == 0, f"{what}: {bad[0].size} entries off, worst {err.max():.3e} at {np.argmax(err)}"


def run_Ax(dg, x):
    xt = torch.from_numpy(x).cuda()
    y = torch.full_like(xt, float("nan"))
    bvg.bvg_spmv_Ax(dg, xt, y)
    bvg.bvg_device_check(dg)
    return y.cpu().numpy()


def traced(dg, fn):
    bvg.bvg_trace_enable(dg, True)
    bvg.bvg_trace_read(dg)
    fn()
    tr = bvg.bvg_trace_read(dg)
    bvg.bvg_trace_enable(dg, False)
    return set(tr)


@pytest.mark.parametrize("name", ["tiny_web", "ragged_1037", "web_50k"])
def test_default_is_one_launch(name):
    g, hg, dg, ref = graph(name)
    assert traced(dg, lambda: run_Ax(dg, synth.rhs(g.n, 1, 3))) == {"pull_fused"}


def test_long_runs_keep_two_launches():
    """Runs of up to 900 ids make some row tiles' x windows wider than the
    kernel holds: that graph keeps the two-launch pull (its parity with the
    oracle is in test_pull_fused_matches_oracle)."""
    g, hg, dg, ref = graph("long_runs")
    tr = traced(dg, lambda: run_Ax(dg, synth.rhs(g.n, 1, 3)))
    assert "pull_fused" not in tr and {"pull_items", "pull_rows"} <= tr


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("kind", ["uniform", "signed", "wide"])
def test_pull_fused_matches_oracle(name, kind):
    g, hg, dg, ref = graph(name)
    x = synth.input_kind(kind, g.n, 1, synth.seed_for(8, 200 + len(kind)))
    x64 = x.astype(np.float64)
    check_close(run_Ax(dg, x), oracle.csr_Ax(g.row_ptr, g.col, x64),
                oracle.bv_Ax(g.row_ptr, g.col, ref, x64, absval=True), f"pull fused {kind} {name}")


@pytest.mark.parametrize("name", ["tiny_web", "ragged_1037", "web_50k"])
def test_pull_fused_is_the_exact_sum_rounded_once(name):
    g, hg, dg, ref = graph(name)
    x = (np.float64(2.0 ** -10) + (1 - 2.0 ** -10) * synth.uniform(g.n, synth.seed_for(8, 210))).astype(np.float32)
    got = run_Ax(dg, x.reshape(-1, 1))[:, 0]
    want32 = oracle.csr_Ax(g.row_ptr, g.col, x.astype(np.float64).reshape(-1, 1))[:, 0].astype(np.float32)
    d = np.abs(got.view(np.int32).astype(np.int64) - want32.view(np.int32).astype(np.int64))
    assert d.max() <= 1, d.max()
    assert np.mean(d == 0) >= 0.999, np.mean(d == 0)


def test_pull_fused_signed_dyadic_bit_exact():
    for name in GRAPHS:
        g, hg, dg, ref = graph(name)
        x = synth.signed_dyadic_rhs(g.n, 1, synth.seed_for(8, 220))
        np.testing.assert_array_equal(run_Ax(dg, x).astype(np.float64), oracle.csr_Ax(g.row_ptr, g.col, x))


def test_pull_fused_against_two_kernels_and_deterministic():
    g, hg, dg, ref = graph("web_50k")
    x = synth.signed_rhs(g.n, 1, synth.seed_for(8, 230))
    y1, y2 = run_Ax(dg, x), run_Ax(dg, x)
    np.testing.assert_array_equal(y1, y2)
    bvg.bvg_set_config(dg, pull_fused=0)
    try:
        assert traced(dg, lambda: run_Ax(dg, x)) == {"pull_items", "pull_rows"}
        y3 = run_Ax(dg, x)
    finally:
        bvg.bvg_set_config(dg, pull_fused=-1)
    x64 = x.astype(np.float64)
    check_close(y1, y3.astype(np.float64), oracle.bv_Ax(g.row_ptr, g.col, ref, x64, absval=True), "fused vs two")


def test_pull_fused_nonfinite_inputs():
    """A NaN and an infinity in x: the tiles that read them take the
    compensated path; exactly the rows that the compressed formula (the
    oracle's own, Sec. 4) makes non-finite are non-finite, and every other
    row matches the oracle."""
    g, hg, dg, ref = graph("web_50k")
    x = synth.rhs(g.n, 1, synth.seed_for(8, 240))
    x[1234, 0] = np.nan
    x[40000, 0] = np.inf
    got = run_Ax(dg, x)
    x64 = x.astype(np.float64)
    bad = ~np.isfinite(oracle.bv_Ax(g.row_ptr, g.col, ref, x64))
    assert bad.any()
    np.testing.assert_array_equal(~np.isfinite(got), bad)
    mag = oracle.bv_Ax(g.row_ptr, g.col, ref, np.where(np.isfinite(x64), x64, 0.0), absval=True)
    check_close(got[~bad], oracle.csr_Ax(g.row_ptr, g.col, x64)[~bad], mag[~bad], "finite rows")


def test_pull_fused_strided_column():
    """One column of a wider row-major tensor (leading dimension 5)."""
    g, hg, dg, ref = graph("ragged_1037")
    X = torch.from_numpy(synth.signed_rhs(g.n, 5, synth.seed_for(8, 250))).cuda()
    Y = torch.full_like(X, 7.0)
    x, y = X[:, 2:3], Y[:, 2:3]
    assert traced(dg, lambda: bvg.bvg_spmv_Ax(dg, x, y)) == {"pull_fused"}
    x64 = X[:, 2:3].cpu().numpy().astype(np.float64)
    check_close(Y[:, 2:3].cpu().numpy(), oracle.csr_Ax(g.row_ptr, g.col, x64),
                oracle.bv_Ax(g.row_ptr, g.col, ref, x64, absval=True), "strided")
    assert np.all(np.delete(Y.cpu().numpy(), 2, axis=1) == 7.0)  # the other columns untouched


def test_pull_fused_not_used_on_random_ids():
    """Rows whose entries lie far from the row (random ids) keep the
    two-kernel pull, which matches the oracle."""
    g = synth.copying_model(synth.replace(synth.social_5m4(), n=20_000))
    hg = bvg.bvg_encode(g.row_ptr, g.col)
    ref, _ = bvg.bvg_get_refs(hg)
    dg = bvg.bvg_upload(hg)
    x = synth.rhs(g.n, 1, 5)
    assert traced(dg, lambda: run_Ax(dg, x)) == {"pull_items", "pull_rows"}
    x64 = x.astype(np.float64)
    check_close(run_Ax(dg, x), oracle.csr_Ax(g.row_ptr, g.col, x64),
                oracle.bv_Ax(g.row_ptr, g.col, ref, x64, absval=True), "social")


def test_pull_fused_full_size():
    """n = 862,664 (the bench's graph): the default pull is one launch and
    matches the oracle on every row, uniform and wide-range x."""
    g = synth.copying_model(synth.web_862k())
    hg = bvg.bvg_encode(g.row_ptr, g.col)
    ref, _ = bvg.bvg_get_refs(hg)
    dg = bvg.bvg_upload(hg)
    for kind in ("uniform", "wide"):
        x = synth.input_kind(kind, g.n, 1, synth.seed_for(8, 260 + len(kind)))
        x64 = x.astype(np.float64)
        check_close(run_Ax(dg, x), oracle.csr_Ax(g.row_ptr, g.col, x64),
                    oracle.bv_Ax(g.row_ptr, g.col, ref, x64, absval=True), f"862k pull {kind}")
    assert traced(dg, lambda: run_Ax(dg, synth.rhs(g.n, 1, 3))) == {"pull_fused"}

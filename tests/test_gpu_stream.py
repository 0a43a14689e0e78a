"""Streamed row blocks (bvg_stream_*): the structure kept in page-locked host
memory and copied block by block through two device slots, at a forced small
budget (many blocks), against the CPU oracle: y = A x^T and y = x A (the
stream built on A^T), element by element at the product tolerance
1e-5 * max(|y*|, s), s computed by the oracle on the stream's own block
references; signed dyadic inputs bit for bit."""
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


def transpose(g):
    rp = np.asarray(g.row_ptr, np.int64)
    ci = np.asarray(g.col, np.int64)
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(rp))
    order = np.lexsort((src, ci))
    tp = np.zeros(g.n + 1, np.int64)
    tp[1:] = np.cumsum(np.bincount(ci, minlength=g.n))
    return synth.Graph(g.n, tp, src[order].astype(np.int32))


def check(got, want, mag, what):
    err = np.abs(got.astype(np.float64) - want)
    bad = ~(err <= RTOL * np.maximum(np.abs(want), mag) + 1e-300)
    assert not bad.any(), f"{what}: {int(bad.sum())} entries off, worst {err.max():.3e}"


GRAPHS = {
    "tiny_web": lambda: synth.copying_model(synth.tiny_web()),
    "social_20k": lambda: synth.copying_model(synth.replace(synth.social_5m4(), n=20_000)),
    "long_runs": lambda: synth.copying_model(synth.GraphSpec(n=5000, seed=6, p_copy=0.6, fidelity=0.95,
                                                             extra_mean=1.0, fresh_mean=300, q_run=0.9,
                                                             run_min=100, run_max=900, gap_mean=50.0)),
}


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("left", [False, True])
def test_stream_products_match_oracle(name, left):
    g = GRAPHS[name]()
    budget = 96 << 10  # 48 KiB per slot: many blocks
    s = bvg.bvg_stream_create(g.row_ptr, g.col, budget, left=left)
    info = bvg.bvg_stream_info(s)
    assert info["blocks"] >= 4 and info["slot_bytes"] <= budget // 2, info
    M = transpose(g) if left else g
    ref = bvg.bvg_stream_get_refs(s)
    assert np.all((ref < 0) | (np.arange(g.n) - ref >= 1)) and np.all((ref < 0) | (np.arange(g.n) - ref <= 7))
    for k in (1, 8, 33, 64):
        for call in range(2):  # a second call reuses the slots
            x = synth.input_kind("signed" if call else "uniform", g.n, k, synth.seed_for(10, k + 100 * call))
            x64 = x.astype(np.float64)
            xt = torch.from_numpy(x).cuda()
            y = torch.full_like(xt, float("nan"))
            bvg.bvg_stream_spmv(s, xt, y)
            want = oracle.csr_Ax(M.row_ptr, M.col, x64)
            mag = oracle.bv_Ax(M.row_ptr, M.col, ref, x64, absval=True)
            check(y.cpu().numpy(), want, mag, f"stream {name} left={left} k={k} call={call}")


def test_stream_dyadic_bit_exact_and_other_stream():
    g = GRAPHS["tiny_web"]()
    for left in (False, True):
        s = bvg.bvg_stream_create(g.row_ptr, g.col, 64 << 10, left=left)
        x = synth.signed_dyadic_rhs(g.n, 4, synth.seed_for(10, 7))
        xt = torch.from_numpy(x).cuda()
        y = torch.empty_like(xt)
        side = torch.cuda.Stream()
        with torch.cuda.stream(side):
            bvg.bvg_stream_spmv(s, xt, y, stream=side)
        side.synchronize()
        want = oracle.csr_xA(g.row_ptr, g.col, x) if left else oracle.csr_Ax(g.row_ptr, g.col, x)
        np.testing.assert_array_equal(y.cpu().numpy().astype(np.float64), want)


def test_stream_one_block_and_invalid_arguments():
    g = GRAPHS["tiny_web"]()
    s = bvg.bvg_stream_create(g.row_ptr, g.col, 1 << 30)
    assert bvg.bvg_stream_info(s)["blocks"] == 1
    x = torch.ones(g.n, device="cuda")
    y = torch.empty_like(x)
    bvg.bvg_stream_spmv(s, x, y)
    np.testing.assert_allclose(y.cpu().numpy(), np.diff(g.row_ptr), rtol=1e-6)  # A 1 = out-degrees
    with pytest.raises(bvg.BvgError) as e:
        bvg.bvg_stream_spmv(s, x, x)
    assert e.value.status == bvg.BVG_ERR_INVALID_ARG
    lib = bvg.load()
    hx = np.ones(g.n, np.float32)
    assert lib.bvg_stream_spmv(s.ptr, hx.ctypes.data, y.data_ptr(), 1, 1, None) == bvg.BVG_ERR_INVALID_ARG

"""The allocation-free x A entry point (bvg_spmv_xA_noalloc), through the C
ABI, against the regular one (bvg_spmv_xA). It exists for callers that may
not allocate device memory once running (their memory belongs to another
allocator's pool, or cudaMalloc's implicit synchronisation is not
acceptable); it keeps its scratch in a fixed device array of 4,194,304 floats.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test; it also passes on its own."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1708_07271_gb300 as bvg  # noqa: E402

RTOL = 1e-5  # the per-entry tolerance of the product parity tests


def within_tolerance(got, want, mag):
    err = np.abs(got.astype(np.float64) - want.astype(np.float64))
    return bool(np.all(err <= RTOL * np.maximum(np.abs(want), mag) + 1e-30))


@pytest.mark.parametrize("k", [1, 3, 8])
def test_noalloc_matches_regular_entry_point_twice(k):
    g = synth.copying_model(synth.tiny_web())
    hg = bvg.bvg_encode(g.row_ptr, g.col)
    ref, _ = bvg.bvg_get_refs(hg)
    dg = bvg.bvg_upload(hg)
    lib = bvg.load()
    for call in range(2):  # two calls in a row share the fixed scratch
        x = synth.rhs(g.n, k, 4000 + 10 * k + call)
        xt = torch.from_numpy(x).cuda()
        y_reg = torch.full_like(xt, float("nan"))
        y_na = torch.full_like(xt, float("nan"))
        bvg.bvg_spmv_xA(dg, xt, y_reg)
        rc = lib.bvg_spmv_xA_noalloc(dg.ptr, xt.data_ptr(), y_na.data_ptr(), k, k,
                                     torch.cuda.current_stream().cuda_stream)
        assert rc == bvg.BVG_OK, bvg.load().bvg_last_error()
        torch.cuda.synchronize()
        mag = np.abs(oracle.bv_xA(g.row_ptr, g.col, ref, x.astype(np.float64), absval=True))
        assert within_tolerance(y_na.cpu().numpy(), y_reg.cpu().numpy(), mag), f"call {call}"
        assert not torch.isnan(y_na).any()


def test_noalloc_rejects_graphs_beyond_its_scratch():
    n = (1 << 22) + 1
    g = synth.Graph(n, np.zeros(n + 1, np.int64), np.zeros(0, np.int32))
    dg = bvg.bvg_upload(bvg.bvg_encode(g.row_ptr, g.col))
    x = torch.zeros(n, device="cuda")
    y = torch.zeros(n, device="cuda")
    with pytest.raises(bvg.BvgError) as e:
        bvg.bvg_spmv_xA_noalloc(dg, x, y)
    assert e.value.status == bvg.BVG_ERR_UNSUPPORTED


def _noalloc(dg, x, y, k, ld):
    return bvg.load().bvg_spmv_xA_noalloc(dg.ptr, x, y, k, ld, torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("k", [16, 32, 48])
def test_noalloc_wide_blocks_against_oracle(k):
    """k = 16, 32, 48 on the 10,000-row graph (column blocks of 16 and 32, the
    widest the fixed scratch allows there): every entry against the oracle,
    and the regular entry point within the same tolerance, twice in a row."""
    g = synth.copying_model(synth.tiny_web())
    hg = bvg.bvg_encode(g.row_ptr, g.col)
    ref, _ = bvg.bvg_get_refs(hg)
    dg = bvg.bvg_upload(hg)
    for call in range(2):
        x = synth.rhs(g.n, k, 4100 + k + call)
        x64 = x.astype(np.float64)
        xt = torch.from_numpy(x).cuda()
        y = torch.full_like(xt, float("nan"))
        assert _noalloc(dg, xt.data_ptr(), y.data_ptr(), k, k) == bvg.BVG_OK, bvg.load().bvg_last_error()
        torch.cuda.synchronize()
        mag = oracle.bv_xA(g.row_ptr, g.col, ref, x64, absval=True)
        assert within_tolerance(y.cpu().numpy(), oracle.csr_xA(g.row_ptr, g.col, x64), mag), f"call {call}"
        y_reg = torch.empty_like(xt)
        bvg.bvg_spmv_xA(dg, xt, y_reg)
        assert within_tolerance(y.cpu().numpy(), y_reg.cpu().numpy(), mag)


@pytest.mark.parametrize("col0", [0, 1])
def test_noalloc_scratch_limited_blocks_and_padded_stride(col0):
    """n = 200,000: the fixed scratch holds 20 columns of z, so column blocks
    shrink to 16; k = 33 taken as a column slice of an n x 40 tensor (ld = 40,
    starting at column 0 for 128-bit loads or at column 1 for scalar loads):
    every entry against the oracle and the regular entry point, and the
    columns outside the slice are left untouched."""
    g = synth.copying_model(synth.web_small(200_000, synth.seed_for(7, 1)))
    hg = bvg.bvg_encode(g.row_ptr, g.col)
    ref, _ = bvg.bvg_get_refs(hg)
    dg = bvg.bvg_upload(hg)
    k, ld = 33, 40
    X = torch.from_numpy(synth.rhs(g.n, ld, synth.seed_for(7, 2))).cuda()
    Y = torch.full((g.n, ld), 7.0, device="cuda")
    x, y = X[:, col0:col0 + k], Y[:, col0:col0 + k]
    for call in range(2):
        y.fill_(float("nan"))
        assert _noalloc(dg, x.data_ptr(), y.data_ptr(), k, ld) == bvg.BVG_OK, bvg.load().bvg_last_error()
        torch.cuda.synchronize()
        x64 = x.cpu().numpy().astype(np.float64)
        mag = oracle.bv_xA(g.row_ptr, g.col, ref, x64, absval=True)
        assert within_tolerance(y.cpu().numpy(), oracle.csr_xA(g.row_ptr, g.col, x64), mag), f"call {call}"
        y_reg = torch.empty(g.n, ld, device="cuda")[:, col0:col0 + k]  # the same strides as x
        bvg.bvg_spmv_xA(dg, x, y_reg)
        assert within_tolerance(y.cpu().numpy(), y_reg.cpu().numpy(), mag)
    outside = torch.cat([Y[:, :col0], Y[:, col0 + k:]], dim=1)
    assert (outside == 7.0).all()


def test_noalloc_rejects_host_pointers():
    """A host buffer given for x or y is refused with BVG_ERR_INVALID_ARG
    before any kernel is launched."""
    g = synth.copying_model(synth.tiny_web())
    dg = bvg.bvg_upload(bvg.bvg_encode(g.row_ptr, g.col))
    hx = np.ones(g.n, np.float32)
    hy = np.zeros(g.n, np.float32)
    xd = torch.ones(g.n, device="cuda")
    yd = torch.zeros(g.n, device="cuda")
    assert _noalloc(dg, hx.ctypes.data, yd.data_ptr(), 1, 1) == bvg.BVG_ERR_INVALID_ARG
    assert _noalloc(dg, xd.data_ptr(), hy.ctypes.data, 1, 1) == bvg.BVG_ERR_INVALID_ARG
    assert np.all(hy == 0)

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

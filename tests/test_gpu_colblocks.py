"""Products over column blocks (Sec. 6, future work: A split into
submatrices of consecutive columns, each encoded with its own references)
through the C ABI against the CPU oracle: x A (each block's product gives
the columns of its range) and A x^T (the blocks' products added), on graphs
whose rows link into two regions of ids, with 1, 2 and 3 blocks (one cut
off the region boundary). Tolerance per entry: 1e-5 * max(|y*|, s), s the
sum over blocks of the oracle's magnitudes on each block's own A'; dyadic
inputs bit-exact."""
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
GRAPHS = {"two_region_6000": (3000, 5), "two_region_2074": (1037, 7)}
_cache = {}


def graph(name):
    if name not in _cache:
        _cache[name] = synth.two_region(*GRAPHS[name])
    return _cache[name]


def cuts_for(n, nb):
    # 2a, 3a: bounds on whole 1024-column tiles (the one-vector x A runs just
    # each block's tiles into y); 2, 3: the product of each block into
    # scratch, then its rows copied
    return {"1": [0, n], "2": [0, n // 2, n], "3": [0, n // 3, n // 2 + 17, n],
            "2a": [0, 2048, n], "3a": [0, 1024, 2048, n]}[nb]


def magnitude(g, cuts, x64, left):
    s = 0.0
    for rp, ci in bvg.split_columns(g.row_ptr, g.col, cuts):
        ref, _ = bvg.bvg_get_refs(bvg.bvg_encode(rp, ci))
        s = s + (oracle.bv_xA(rp, ci, ref, x64, absval=True) if left else oracle.bv_Ax(rp, ci, ref, x64, absval=True))
    return s


def check_close(got, want, mag, what):
    err = np.abs(got.astype(np.float64) - want)
    bad = np.nonzero(~(err <= RTOL * np.maximum(np.abs(want), mag) + 1e-300))
    assert bad[0].size == 0, f"{what}: {bad[0].size} entries off, worst {err.max():.3e}"


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("nb", ["1", "2", "3", "2a", "3a"])
@pytest.mark.parametrize("k", [1, 8])
def test_colblock_products_match_oracle(name, nb, k):
    g = graph(name)
    cuts = cuts_for(g.n, nb)
    cb = bvg.bvg_colblocks_create(g.row_ptr, g.col, cuts=cuts)
    for kind in ("uniform", "signed"):
        x = synth.input_kind(kind, g.n, k, synth.seed_for(9, 3 + k))
        x64 = x.astype(np.float64)
        xt = torch.from_numpy(x).cuda()
        for left in (True, False):
            ys = []
            for _ in range(2):  # two calls in a row: the same result
                y = torch.full_like(xt, float("nan"))
                (bvg.bvg_spmv_xA_colblocks if left else bvg.bvg_spmv_Ax_colblocks)(cb, xt, y)
                ys.append(y.cpu().numpy())
            np.testing.assert_array_equal(ys[0], ys[1])
            want = oracle.csr_xA(g.row_ptr, g.col, x64) if left else oracle.csr_Ax(g.row_ptr, g.col, x64)
            check_close(ys[0], want, magnitude(g, cuts, x64, left), f"{name} nb={nb} k={k} {kind} left={left}")


def test_colblock_dyadic_bit_exact():
    g = graph("two_region_6000")
    cb = bvg.bvg_colblocks_create(g.row_ptr, g.col, nblocks=3)
    x = synth.signed_dyadic_rhs(g.n, 4, synth.seed_for(9, 20))
    xt = torch.from_numpy(x).cuda()
    for left, f, ref in ((True, bvg.bvg_spmv_xA_colblocks, oracle.csr_xA), (False, bvg.bvg_spmv_Ax_colblocks, oracle.csr_Ax)):
        y = torch.empty_like(xt)
        f(cb, xt, y)
        np.testing.assert_array_equal(y.cpu().numpy().astype(np.float64), ref(g.row_ptr, g.col, x.astype(np.float64)))


def test_colblock_invalid_arguments():
    g = graph("two_region_2074")
    cb = bvg.bvg_colblocks_create(g.row_ptr, g.col, nblocks=2)
    x = torch.zeros(g.n, device="cuda")
    y = torch.zeros(g.n, device="cuda")
    bad = bvg.ColumnBlocks(cb.n, [0, 5, g.n - 1], cb.hosts, cb.devs)  # cuts do not reach n
    with pytest.raises(bvg.BvgError) as e:
        bvg.bvg_spmv_xA_colblocks(bad, x, y)
    assert e.value.status == bvg.BVG_ERR_INVALID_ARG
    with pytest.raises(bvg.BvgError) as e:
        bvg.bvg_spmv_Ax_colblocks(cb, x, y, scratch=y)  # scratch aliases y
    assert e.value.status == bvg.BVG_ERR_INVALID_ARG

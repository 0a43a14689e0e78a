"""Row shards on the GPU: the masked encodings of contiguous row blocks give,
through the CUDA path, the block's rows of A x^T and partial sums of x A that
add up to the full product (the exchange itself runs on CPU ranks in
test_shard_gloo.py; this pool has one GPU per run)."""
import numpy as np
import pytest

import oracle
import synth
from paper_1708_07271_gb300 import shard

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1708_07271_gb300 as bvg  # noqa: E402


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("k", [1, 8])
def test_masked_blocks_sum_to_the_product(world, k):
    g = synth.copying_model(synth.tiny_web())
    x = synth.rhs(g.n, k, synth.seed_for(60, k))
    x64 = x.astype(np.float64)
    xt = torch.from_numpy(x).cuda()
    ax = np.zeros_like(x64)
    xa = np.zeros_like(x64)
    for a, b in shard.row_blocks(g.row_ptr, world):
        rp, ci = shard.masked_csr(g.row_ptr, g.col, a, b)
        dg = bvg.bvg_upload(bvg.bvg_encode(rp, ci))
        y = torch.full_like(xt, float("nan"))
        bvg.bvg_spmv_Ax(dg, xt, y)
        ax[a:b] = y.cpu().numpy().astype(np.float64)[a:b]
        bvg.bvg_spmv_xA(dg, xt, y)
        xa += y.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(ax, oracle.csr_Ax(g.row_ptr, g.col, x64), rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(xa, oracle.csr_xA(g.row_ptr, g.col, x64), rtol=1e-5, atol=1e-5)

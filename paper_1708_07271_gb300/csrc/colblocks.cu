// Products over A split into submatrices of consecutive columns (Sec. 6,
// future work: with the window applied per block, a reference need only
// match the part of a row inside one block). A = sum_b A_b, where A_b keeps
// A's entries in columns [cuts[b], cuts[b+1]); each A_b is encoded and
// uploaded on its own (n rows, the same ids), so every block chooses its own
// references.
//   x A: block b's product is zero outside its columns, so y takes rows
//        [cuts[b], cuts[b+1]) of block b's product: for one right-hand side
//        with block bounds on whole 1024-column tiles, one launch runs every
//        block's own tiles of the one-vector kernel (the blocks' arguments
//        in the launch's parameters), each CTA a tile of its block, into y;
//        otherwise each block's product goes to scratch and its rows are
//        copied;
//   A x^T: y = sum_b A_b x^T, the blocks' products added in block order.
#include <cuda_runtime.h>

#include <algorithm>

#include "bvg_internal.h"
#include "fused.cuh"

namespace bvg {

// Blocks one launch serves: their one-vector kernel arguments (fa[b].tile0 =
// the first tile of block b's columns) and the CTAs of each block.
constexpr int kMaxColBlocks = 16;
struct FxBlocks {
    FxArgs fa[kMaxColBlocks];
    int64_t cta_end[kMaxColBlocks];  // CTAs [cta_end[b - 1], cta_end[b]) run block b's tiles
    int32_t nb;
};

__global__ void __launch_bounds__(kFxNT, 6) k_push_fx_blocks(const __grid_constant__ FxBlocks fb) {
    __shared__ __align__(16) FxSmem S;
    int b = 0;
    for (int i = 1; i < fb.nb; i++)
        if ((int64_t)blockIdx.x >= fb.cta_end[i - 1]) b = i;
    const int64_t first = b ? fb.cta_end[b - 1] : 0;
    const FxArgs& fa = fb.fa[b];
    PrArgs pa{};
    fx_tile<0>(fa.tile0 + ((int64_t)blockIdx.x - first), fa, pa, S);
}

// y += s over n rows of k values (leading dimension ld).
__global__ void k_add_rows(float* __restrict__ y, const float* __restrict__ s, int64_t n, int32_t k, int64_t ld) {
    const int64_t total = n * (int64_t)k;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / k, c = t % k;
        y[i * ld + c] = __fadd_rn(y[i * ld + c], s[i * ld + c]);
    }
}

static int check_blocks(const bvg_dev_graph* const* blocks, int32_t nblocks, const float* x, const float* y,
                        const float* scratch, int32_t k, int64_t ld, const char* what) {
    if (!blocks || nblocks < 1) return fail(BVG_ERR_INVALID_ARG, "%s: need at least one block", what);
    if (k < 1 || ld < k) return fail(BVG_ERR_INVALID_ARG, "%s: need k >= 1 and ld >= k", what);
    for (int32_t b = 0; b < nblocks; b++) {
        if (!blocks[b]) return fail(BVG_ERR_INVALID_ARG, "%s: NULL block %d", what, b);
        if (blocks[b]->n != blocks[0]->n) return fail(BVG_ERR_INVALID_ARG, "%s: blocks of different n", what);
        if (blocks[b]->device != blocks[0]->device)
            return fail(BVG_ERR_INVALID_ARG, "%s: blocks on different devices", what);
    }
    if (blocks[0]->n == 0) return BVG_OK;
    int rc;
    if ((rc = check_vec(blocks[0], x, "x")) || (rc = check_vec(blocks[0], y, "y"))) return rc;
    if (nblocks > 1 && (rc = check_vec(blocks[0], scratch, "scratch"))) return rc;
    if (x == y || (nblocks > 1 && (scratch == x || scratch == y)))
        return fail(BVG_ERR_INVALID_ARG, "%s: x, y and scratch must not alias", what);
    return BVG_OK;
}

}  // namespace bvg

using namespace bvg;

extern "C" int bvg_spmv_xA_colblocks(const bvg_dev_graph* const* blocks, const int64_t* cuts, int32_t nblocks,
                                     const float* x, float* y, float* scratch, int32_t k, int64_t ld, void* stream) {
    int rc = check_blocks(blocks, nblocks, x, y, scratch, k, ld, "bvg_spmv_xA_colblocks");
    if (rc) return rc;
    const int64_t n = blocks[0]->n;
    if (!cuts || cuts[0] != 0 || cuts[nblocks] != n)
        return fail(BVG_ERR_INVALID_ARG, "bvg_spmv_xA_colblocks: cuts must run from 0 to n");
    for (int32_t b = 0; b < nblocks; b++)
        if (cuts[b + 1] < cuts[b]) return fail(BVG_ERR_INVALID_ARG, "bvg_spmv_xA_colblocks: cuts must not decrease");
    if (n == 0) return BVG_OK;
    if (nblocks == 1) return bvg_spmv_xA(blocks[0], x, y, k, ld, stream);
    cudaStream_t st = (cudaStream_t)stream;
    // one vector, every block served by the one-vector kernel, bounds on whole
    // tiles: one launch over all blocks' tiles
    bool one = k == 1 && ld == 1 && nblocks <= kMaxColBlocks;
    for (int32_t b = 0; one && b < nblocks; b++)
        one = use_fused(blocks[b], 1) && cuts[b] % kFxT == 0 && (cuts[b + 1] % kFxT == 0 || cuts[b + 1] == n);
    if (one) {
        FxBlocks fb{};
        fb.nb = nblocks;
        int64_t ctas = 0;
        for (int32_t b = 0; b < nblocks; b++) {
            fb.fa[b] = fused_args(blocks[b], x, 1, nullptr, y, 1);
            fb.fa[b].tile0 = cuts[b] / kFxT;
            ctas += cuts[b + 1] > cuts[b] ? (cuts[b + 1] + kFxT - 1) / kFxT - cuts[b] / kFxT : 0;
            fb.cta_end[b] = ctas;
        }
        if (ctas > 0) k_push_fx_blocks<<<(unsigned)ctas, kFxNT, 0, st>>>(fb);
        BVG_CUDA_TRY(cudaGetLastError());
        return BVG_OK;
    }
    for (int32_t b = 0; b < nblocks; b++) {
        const int64_t rows = cuts[b + 1] - cuts[b];
        if (rows == 0) continue;
        // one vector, whole column tiles: the block's own tiles write y
        if (k == 1 && ld == 1 && (rc = spmv_xA_columns(blocks[b], x, y, cuts[b], cuts[b + 1], stream)) != BVG_ERR_UNSUPPORTED) {
            if (rc) return rc;
            continue;
        }
        if ((rc = bvg_spmv_xA(blocks[b], x, scratch, k, ld, stream))) return rc;
        BVG_CUDA_TRY(cudaMemcpy2DAsync(y + cuts[b] * ld, (size_t)ld * sizeof(float), scratch + cuts[b] * ld,
                                       (size_t)ld * sizeof(float), (size_t)k * sizeof(float), (size_t)rows,
                                       cudaMemcpyDeviceToDevice, st));
    }
    return BVG_OK;
}

extern "C" int bvg_spmv_Ax_colblocks(const bvg_dev_graph* const* blocks, int32_t nblocks, const float* x, float* y,
                                     float* scratch, int32_t k, int64_t ld, void* stream) {
    int rc = check_blocks(blocks, nblocks, x, y, scratch, k, ld, "bvg_spmv_Ax_colblocks");
    if (rc) return rc;
    const int64_t n = blocks[0]->n;
    if (n == 0) return BVG_OK;
    if ((rc = bvg_spmv_Ax(blocks[0], x, y, k, ld, stream))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t total = n * (int64_t)k;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
    for (int32_t b = 1; b < nblocks; b++) {
        if ((rc = bvg_spmv_Ax(blocks[b], x, scratch, k, ld, stream))) return rc;
        k_add_rows<<<grid, 256, 0, st>>>(y, scratch, n, k, ld);
        BVG_CUDA_TRY(cudaGetLastError());
    }
    return BVG_OK;
}

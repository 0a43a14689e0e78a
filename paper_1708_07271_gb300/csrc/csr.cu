// Plain CSR baseline: the product with the uncompressed pattern of A (the
// comparison of Sec. 5, A against A'), pattern-only (no value array: A is
// binary). y = A x^T uses the CSR of A; y = x A the CSR of A^T.
#include <algorithm>
#include <new>
#include <vector>

#include "device_common.cuh"

using namespace bvg;

namespace bvg {

// A group of G*S lanes owns one row: S parts split the row's entries, each
// lane of a part owns V of the KB right-hand sides. FP32 accumulation.
template <int KB, int V, int S>
__global__ void __launch_bounds__(256) k_csr(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                             const float* __restrict__ x, int64_t ldx, float* __restrict__ y,
                                             int64_t ldy, int64_t n) {
    constexpr int G = KB / V;
    constexpr int GS = G * S;
    const int lg = threadIdx.x % GS;
    const int slice = lg % G, part = lg / G;
    const int64_t rows_per_block = blockDim.x / GS;
    // The loop bound is uniform per warp (its first row), so every lane of a
    // warp reaches the shuffles; lanes past the last row do no work.
    const int64_t warp_first = (int64_t)blockIdx.x * rows_per_block + (threadIdx.x & ~31) / GS;
    const int64_t stride = (int64_t)gridDim.x * rows_per_block;
    for (int64_t w0 = warp_first; w0 < n; w0 += stride) {
        const int64_t i = w0 + (threadIdx.x & 31) / GS;
        const bool valid = i < n;
        float acc[V];
#pragma unroll
        for (int v = 0; v < V; v++) acc[v] = 0.f;
        if (valid) {
            const int64_t e1 = __ldg(rp + i + 1);
            for (int64_t e = __ldg(rp + i) + part; e < e1; e += S) {
                Vec<V> xv = ldv<V>(x + (int64_t)__ldg(ci + e) * ldx + slice * V);
#pragma unroll
                for (int v = 0; v < V; v++) acc[v] += xv.v[v];
            }
        }
#pragma unroll
        for (int v = 0; v < V; v++)
            for (int o = G; o < GS; o <<= 1) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], o);
        if (valid && part == 0) {
            Vec<V> out;
#pragma unroll
            for (int v = 0; v < V; v++) out.v[v] = acc[v];
            stv<V>(y + i * ldy + slice * V, out);
        }
    }
}

template <int KB, int V>
static void launch_csr(const int64_t* rp, const int32_t* ci, int64_t n, const float* x, int64_t ldx, float* y,
                       int64_t ldy, cudaStream_t st) {
    constexpr int G = KB / V;
    constexpr int S = G >= 8 ? 1 : 8 / G;
    const int64_t rows_per_block = 256 / (G * S);
    int64_t grid = (n + rows_per_block - 1) / rows_per_block;
    grid = std::min<int64_t>(grid, 152 * 64);
    k_csr<KB, V, S><<<(unsigned)std::max<int64_t>(grid, 1), 256, 0, st>>>(rp, ci, x, ldx, y, ldy, n);
}

static int block_k(int64_t r) {
    int kb = 32;
    while (kb > r) kb >>= 1;
    return kb;
}

static int pick_v(int kb, int64_t ld, int64_t col, const void* a, const void* b) {
    auto ok = [&](int v) {
        if (kb % v || ld % v || col % v) return false;
        for (const void* p : {a, b})
            if (((uintptr_t)((const float*)p + col) % (4 * v))) return false;
        return true;
    };
    if (kb >= 4 && ok(4)) return 4;
    if (kb == 2 && ok(2)) return 2;
    return 1;
}

static int csr_product(const int64_t* rp, const int32_t* ci, int64_t n, const float* x, float* y, int32_t k,
                       int64_t ld, void* stream, const char* who) {
    if (k < 1 || ld < k || !x || !y) return fail(BVG_ERR_INVALID_ARG, "%s: bad k/ld or NULL vector", who);
    if ((uintptr_t)x % 4 || (uintptr_t)y % 4) return fail(BVG_ERR_INVALID_ARG, "%s: misaligned vector", who);
    if (n == 0) return BVG_OK;
    cudaStream_t st = (cudaStream_t)stream;
    for (int64_t c0 = 0; c0 < k;) {
        const int kb = block_k(k - c0);
        const int v = pick_v(kb, ld, c0, x, y);
        switch (kb * 8 + v) {
            case 1 * 8 + 1: launch_csr<1, 1>(rp, ci, n, x + c0, ld, y + c0, ld, st); break;
            case 2 * 8 + 1: launch_csr<2, 1>(rp, ci, n, x + c0, ld, y + c0, ld, st); break;
            case 2 * 8 + 2: launch_csr<2, 2>(rp, ci, n, x + c0, ld, y + c0, ld, st); break;
            case 4 * 8 + 1: launch_csr<4, 1>(rp, ci, n, x + c0, ld, y + c0, ld, st); break;
            case 4 * 8 + 4: launch_csr<4, 4>(rp, ci, n, x + c0, ld, y + c0, ld, st); break;
            case 8 * 8 + 1: launch_csr<8, 1>(rp, ci, n, x + c0, ld, y + c0, ld, st); break;
            case 8 * 8 + 4: launch_csr<8, 4>(rp, ci, n, x + c0, ld, y + c0, ld, st); break;
            case 16 * 8 + 1: launch_csr<16, 1>(rp, ci, n, x + c0, ld, y + c0, ld, st); break;
            case 16 * 8 + 4: launch_csr<16, 4>(rp, ci, n, x + c0, ld, y + c0, ld, st); break;
            case 32 * 8 + 1: launch_csr<32, 1>(rp, ci, n, x + c0, ld, y + c0, ld, st); break;
            case 32 * 8 + 4: launch_csr<32, 4>(rp, ci, n, x + c0, ld, y + c0, ld, st); break;
            default: return fail(BVG_ERR_INVALID_ARG, "%s: no kernel for kb=%d v=%d", who, kb, v);
        }
        c0 += kb;
    }
    BVG_CUDA_TRY(cudaGetLastError());
    return BVG_OK;
}

}  // namespace bvg

extern "C" int bvg_csr_upload(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, void* stream,
                              bvg_csr_graph** out) {
    if (!out || n < 0 || !row_ptr) return fail(BVG_ERR_INVALID_ARG, "bvg_csr_upload: bad argument");
    *out = nullptr;
    if (row_ptr[0] != 0) return fail(BVG_ERR_BAD_GRAPH, "bvg_csr_upload: row_ptr[0] != 0");
    const int64_t m = row_ptr[n];
    for (int64_t i = 0; i < n; i++) {
        if (row_ptr[i + 1] < row_ptr[i]) return fail(BVG_ERR_BAD_GRAPH, "bvg_csr_upload: row_ptr decreases");
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++)
            if (col_idx[e] < 0 || col_idx[e] >= n || (e > row_ptr[i] && col_idx[e - 1] >= col_idx[e]))
                return fail(BVG_ERR_BAD_GRAPH, "bvg_csr_upload: bad id in row %lld", (long long)i);
    }
    bvg_csr_graph* g = new (std::nothrow) bvg_csr_graph();
    if (!g) return fail(BVG_ERR_OOM, "bvg_csr_upload: host allocation failed");
    std::vector<int64_t> rpt(n + 1, 0);
    std::vector<int32_t> cit(m);
    for (int64_t e = 0; e < m; e++) rpt[col_idx[e] + 1]++;
    for (int64_t j = 0; j < n; j++) rpt[j + 1] += rpt[j];
    {
        std::vector<int64_t> fill(rpt.begin(), rpt.end() - 1);
        for (int64_t i = 0; i < n; i++)
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++) cit[fill[col_idx[e]]++] = (int32_t)i;
    }
    cudaStream_t st = (cudaStream_t)stream;
    g->n = n;
    g->m = m;
    cudaGetDevice(&g->device);
    auto alloc_copy = [&](void** dst, const void* src, size_t bytes) -> int {
        cudaError_t e = cudaMalloc(dst, bytes ? bytes : 16);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(BVG_ERR_OOM, "bvg_csr_upload: cudaMalloc failed");
        }
        if (bytes && cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return fail(BVG_ERR_CUDA, "bvg_csr_upload: copy failed");
        return BVG_OK;
    };
    int rc;
    if ((rc = alloc_copy((void**)&g->rp, row_ptr, (n + 1) * sizeof(int64_t))) ||
        (rc = alloc_copy((void**)&g->ci, col_idx, m * sizeof(int32_t))) ||
        (rc = alloc_copy((void**)&g->rpt, rpt.data(), (n + 1) * sizeof(int64_t))) ||
        (rc = alloc_copy((void**)&g->cit, cit.data(), m * sizeof(int32_t)))) {
        bvg_free_csr(g);
        return rc;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        bvg_free_csr(g);
        return fail(BVG_ERR_CUDA, "bvg_csr_upload: synchronize failed");
    }
    *out = g;
    return BVG_OK;
}

extern "C" int bvg_csr_spmv_Ax(const bvg_csr_graph* g, const float* x, float* y, int32_t k, int64_t ld,
                               void* stream) {
    if (!g) return fail(BVG_ERR_INVALID_ARG, "bvg_csr_spmv_Ax: NULL graph");
    return csr_product(g->rp, g->ci, g->n, x, y, k, ld, stream, "bvg_csr_spmv_Ax");
}

extern "C" int bvg_csr_spmv_xA(const bvg_csr_graph* g, const float* x, float* y, int32_t k, int64_t ld,
                               void* stream) {
    if (!g) return fail(BVG_ERR_INVALID_ARG, "bvg_csr_spmv_xA: NULL graph");
    return csr_product(g->rpt, g->cit, g->n, x, y, k, ld, stream, "bvg_csr_spmv_xA");
}

extern "C" void bvg_free_csr(bvg_csr_graph* g) {
    if (!g) return;
    if (g->rp) cudaFree(g->rp);
    if (g->ci) cudaFree(g->ci);
    if (g->rpt) cudaFree(g->rpt);
    if (g->cit) cudaFree(g->cit);
    delete g;
}

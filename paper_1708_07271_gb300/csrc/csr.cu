// Plain CSR baseline: the product with the uncompressed pattern of A (the
// comparison of Sec. 5, A against A'), pattern-only (no value array: A is
// binary). y = A x^T uses the CSR of A; y = x A the CSR of A^T.
#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include <cusparse.h>

#include "device_common.cuh"

using namespace bvg;

namespace bvg {

// Rows longer than this are summed by a whole CTA (k_csr_hub): with a few
// lanes per row, one row of 200,000 entries (a hub of a power-law graph)
// would hold up the whole product.
constexpr int64_t kCsrHub = 2048;

// A group of G*S lanes owns one row: S parts split the row's entries, each
// lane of a part owns V of the KB right-hand sides. FP32 accumulation. Hub
// rows are skipped (k_csr_hub writes them).
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
        bool hub = false;
        if (valid) {
            const int64_t e0 = __ldg(rp + i), e1 = __ldg(rp + i + 1);
            hub = e1 - e0 > kCsrHub;
            for (int64_t e = e0 + part; e < e1 && !hub; e += S) {
                Vec<V> xv = ldv<V>(x + (int64_t)__ldg(ci + e) * ldx + slice * V);
#pragma unroll
                for (int v = 0; v < V; v++) acc[v] += xv.v[v];
            }
        }
#pragma unroll
        for (int v = 0; v < V; v++)
            for (int o = G; o < GS; o <<= 1) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], o);
        if (valid && !hub && part == 0) {
            Vec<V> out;
#pragma unroll
            for (int v = 0; v < V; v++) out.v[v] = acc[v];
            stv<V>(y + i * ldy + slice * V, out);
        }
    }
}

// One hub row per CTA: the groups of G lanes take the row's entries in
// turn, then the CTA adds the groups' sums in a fixed order (deterministic).
template <int KB, int V>
__global__ void __launch_bounds__(256) k_csr_hub(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                 const int32_t* __restrict__ hub, const float* __restrict__ x,
                                                 int64_t ldx, float* __restrict__ y, int64_t ldy) {
    constexpr int G = KB / V, NG = 256 / G;
    __shared__ float part[NG][KB];
    const int g = threadIdx.x / G, slice = threadIdx.x % G;
    const int64_t i = hub[blockIdx.x];
    float acc[V];
#pragma unroll
    for (int v = 0; v < V; v++) acc[v] = 0.f;
    const int64_t e1 = __ldg(rp + i + 1);
    for (int64_t e = __ldg(rp + i) + g; e < e1; e += NG) {
        Vec<V> xv = ldv<V>(x + (int64_t)__ldg(ci + e) * ldx + slice * V);
#pragma unroll
        for (int v = 0; v < V; v++) acc[v] += xv.v[v];
    }
#pragma unroll
    for (int v = 0; v < V; v++) part[g][slice * V + v] = acc[v];
    __syncthreads();
    for (int c = threadIdx.x; c < KB; c += 256) {
        float t = 0.f;
        for (int q = 0; q < NG; q++) t += part[q][c];
        y[i * ldy + c] = t;
    }
}

template <int KB, int V>
static void launch_csr(const int64_t* rp, const int32_t* ci, const int32_t* hub, int64_t nhub, int64_t n,
                       const float* x, int64_t ldx, float* y, int64_t ldy, cudaStream_t st) {
    constexpr int G = KB / V;
    constexpr int S = G >= 8 ? 1 : 8 / G;
    const int64_t rows_per_block = 256 / (G * S);
    int64_t grid = (n + rows_per_block - 1) / rows_per_block;
    grid = std::min<int64_t>(grid, 152 * 64);
    k_csr<KB, V, S><<<(unsigned)std::max<int64_t>(grid, 1), 256, 0, st>>>(rp, ci, x, ldx, y, ldy, n);
    if (nhub > 0) k_csr_hub<KB, V><<<(unsigned)nhub, 256, 0, st>>>(rp, ci, hub, x, ldx, y, ldy);
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

static int csr_product(const int64_t* rp, const int32_t* ci, const int32_t* hub, int64_t nhub, int64_t n,
                       const float* x, float* y, int32_t k, int64_t ld, void* stream, const char* who) {
    if (k < 1 || ld < k || !x || !y) return fail(BVG_ERR_INVALID_ARG, "%s: bad k/ld or NULL vector", who);
    if ((uintptr_t)x % 4 || (uintptr_t)y % 4) return fail(BVG_ERR_INVALID_ARG, "%s: misaligned vector", who);
    if (n == 0) return BVG_OK;
    cudaStream_t st = (cudaStream_t)stream;
    for (int64_t c0 = 0; c0 < k;) {
        const int kb = block_k(k - c0);
        const int v = pick_v(kb, ld, c0, x, y);
        switch (kb * 8 + v) {
            case 1 * 8 + 1: launch_csr<1, 1>(rp, ci, hub, nhub, n, x + c0, ld, y + c0, ld, st); break;
            case 2 * 8 + 1: launch_csr<2, 1>(rp, ci, hub, nhub, n, x + c0, ld, y + c0, ld, st); break;
            case 2 * 8 + 2: launch_csr<2, 2>(rp, ci, hub, nhub, n, x + c0, ld, y + c0, ld, st); break;
            case 4 * 8 + 1: launch_csr<4, 1>(rp, ci, hub, nhub, n, x + c0, ld, y + c0, ld, st); break;
            case 4 * 8 + 4: launch_csr<4, 4>(rp, ci, hub, nhub, n, x + c0, ld, y + c0, ld, st); break;
            case 8 * 8 + 1: launch_csr<8, 1>(rp, ci, hub, nhub, n, x + c0, ld, y + c0, ld, st); break;
            case 8 * 8 + 4: launch_csr<8, 4>(rp, ci, hub, nhub, n, x + c0, ld, y + c0, ld, st); break;
            case 16 * 8 + 1: launch_csr<16, 1>(rp, ci, hub, nhub, n, x + c0, ld, y + c0, ld, st); break;
            case 16 * 8 + 4: launch_csr<16, 4>(rp, ci, hub, nhub, n, x + c0, ld, y + c0, ld, st); break;
            case 32 * 8 + 1: launch_csr<32, 1>(rp, ci, hub, nhub, n, x + c0, ld, y + c0, ld, st); break;
            case 32 * 8 + 4: launch_csr<32, 4>(rp, ci, hub, nhub, n, x + c0, ld, y + c0, ld, st); break;
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
    std::vector<int32_t> hub, hubt;
    for (int64_t i = 0; i < n; i++) {
        if (row_ptr[i + 1] - row_ptr[i] > kCsrHub) hub.push_back((int32_t)i);
        if (rpt[i + 1] - rpt[i] > kCsrHub) hubt.push_back((int32_t)i);
    }
    int rc;
    if ((rc = alloc_copy((void**)&g->rp, row_ptr, (n + 1) * sizeof(int64_t))) ||
        (rc = alloc_copy((void**)&g->ci, col_idx, m * sizeof(int32_t))) ||
        (rc = alloc_copy((void**)&g->rpt, rpt.data(), (n + 1) * sizeof(int64_t))) ||
        (rc = alloc_copy((void**)&g->cit, cit.data(), m * sizeof(int32_t))) ||
        (rc = alloc_copy((void**)&g->hub, hub.data(), hub.size() * sizeof(int32_t))) ||
        (rc = alloc_copy((void**)&g->hubt, hubt.data(), hubt.size() * sizeof(int32_t)))) {
        bvg_free_csr(g);
        return rc;
    }
    g->nhub = (int64_t)hub.size();
    g->nhubt = (int64_t)hubt.size();
    if (m < ((int64_t)1 << 31)) {  // cuSPARSE with 32-bit indices: row offsets as int32, values 1.0f
        std::vector<int32_t> r32(row_ptr, row_ptr + n + 1), rt32(rpt.begin(), rpt.end());
        std::vector<float> ones((size_t)m, 1.0f);
        if ((rc = alloc_copy((void**)&g->rp32, r32.data(), r32.size() * sizeof(int32_t))) ||
            (rc = alloc_copy((void**)&g->rpt32, rt32.data(), rt32.size() * sizeof(int32_t))) ||
            (rc = alloc_copy((void**)&g->ones, ones.data(), ones.size() * sizeof(float)))) {
            bvg_free_csr(g);
            return rc;
        }
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            bvg_free_csr(g);
            return fail(BVG_ERR_CUDA, "bvg_csr_upload: synchronize failed");
        }
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
    return csr_product(g->rp, g->ci, g->hub, g->nhub, g->n, x, y, k, ld, stream, "bvg_csr_spmv_Ax");
}

extern "C" int bvg_csr_spmv_xA(const bvg_csr_graph* g, const float* x, float* y, int32_t k, int64_t ld,
                               void* stream) {
    if (!g) return fail(BVG_ERR_INVALID_ARG, "bvg_csr_spmv_xA: NULL graph");
    return csr_product(g->rpt, g->cit, g->hubt, g->nhubt, g->n, x, y, k, ld, stream, "bvg_csr_spmv_xA");
}

// ------------------------------------------------------------------ cuSPARSE
namespace {

int sp_fail(cusparseStatus_t s, const char* what) {
    return fail(s == CUSPARSE_STATUS_ALLOC_FAILED ? BVG_ERR_OOM : BVG_ERR_CUDA, "%s: cuSPARSE status %d", what,
                (int)s);
}

#define BVG_SP_TRY(expr, what)                                  \
    do {                                                        \
        cusparseStatus_t s_ = (expr);                           \
        if (s_ != CUSPARSE_STATUS_SUCCESS) return sp_fail(s_, what); \
    } while (0)

// y = M x (M the CSR of A, or of A^T for x A) with cusparseSpMV (k = 1) or
// cusparseSpMM (k > 1, row-major dense blocks of leading dimension ld).
int cusparse_product(bvg_csr_graph* g, bool transpose, const float* x, float* y, int32_t k, int64_t ld,
                     void* stream, const char* who) {
    if (k < 1 || ld < k || !x || !y) return fail(BVG_ERR_INVALID_ARG, "%s: bad k/ld or NULL vector", who);
    if (g->n == 0) return BVG_OK;
    if (!g->ones) return fail(BVG_ERR_UNSUPPORTED, "%s: 2^31 edges or more (32-bit cuSPARSE indices)", who);
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    if (!g->sp_handle) {
        cusparseHandle_t h = nullptr;
        BVG_SP_TRY(cusparseCreate(&h), who);
        g->sp_handle = h;
        cusparseSpMatDescr_t a = nullptr, at = nullptr;
        BVG_SP_TRY(cusparseCreateCsr(&a, g->n, g->n, g->m, g->rp32, g->ci, g->ones, CUSPARSE_INDEX_32I,
                                     CUSPARSE_INDEX_32I, CUSPARSE_INDEX_BASE_ZERO, CUDA_R_32F), who);
        g->sp_mat = a;
        BVG_SP_TRY(cusparseCreateCsr(&at, g->n, g->n, g->m, g->rpt32, g->cit, g->ones, CUSPARSE_INDEX_32I,
                                     CUSPARSE_INDEX_32I, CUSPARSE_INDEX_BASE_ZERO, CUDA_R_32F), who);
        g->sp_matt = at;
    }
    cusparseHandle_t h = (cusparseHandle_t)g->sp_handle;
    cusparseSpMatDescr_t mat = (cusparseSpMatDescr_t)(transpose ? g->sp_matt : g->sp_mat);
    BVG_SP_TRY(cusparseSetStream(h, (cudaStream_t)stream), who);
    const float one = 1.0f, zero = 0.0f;
    size_t need = 0;
    if (k == 1 && ld == 1) {
        cusparseDnVecDescr_t vx = nullptr, vy = nullptr;
        BVG_SP_TRY(cusparseCreateDnVec(&vx, g->n, (void*)x, CUDA_R_32F), who);
        BVG_SP_TRY(cusparseCreateDnVec(&vy, g->n, (void*)y, CUDA_R_32F), who);
        cusparseStatus_t s = cusparseSpMV_bufferSize(h, CUSPARSE_OPERATION_NON_TRANSPOSE, &one, mat, vx, &zero, vy,
                                                     CUDA_R_32F, CUSPARSE_SPMV_ALG_DEFAULT, &need);
        if (s == CUSPARSE_STATUS_SUCCESS && need > g->sp_buf_bytes) {
            cudaStreamSynchronize((cudaStream_t)stream);
            if (g->sp_buf) cudaFree(g->sp_buf);
            g->sp_buf = nullptr;
            g->sp_buf_bytes = 0;
            if (cudaMalloc(&g->sp_buf, need) != cudaSuccess) {
                cudaGetLastError();
                s = CUSPARSE_STATUS_ALLOC_FAILED;
            } else {
                g->sp_buf_bytes = need;
            }
        }
        if (s == CUSPARSE_STATUS_SUCCESS)
            s = cusparseSpMV(h, CUSPARSE_OPERATION_NON_TRANSPOSE, &one, mat, vx, &zero, vy, CUDA_R_32F,
                             CUSPARSE_SPMV_ALG_DEFAULT, g->sp_buf);
        cusparseDestroyDnVec(vx);
        cusparseDestroyDnVec(vy);
        BVG_SP_TRY(s, who);
        return BVG_OK;
    }
    cusparseDnMatDescr_t mx = nullptr, my = nullptr;
    BVG_SP_TRY(cusparseCreateDnMat(&mx, g->n, k, ld, (void*)x, CUDA_R_32F, CUSPARSE_ORDER_ROW), who);
    BVG_SP_TRY(cusparseCreateDnMat(&my, g->n, k, ld, (void*)y, CUDA_R_32F, CUSPARSE_ORDER_ROW), who);
    cusparseStatus_t s = cusparseSpMM_bufferSize(h, CUSPARSE_OPERATION_NON_TRANSPOSE, CUSPARSE_OPERATION_NON_TRANSPOSE,
                                                 &one, mat, mx, &zero, my, CUDA_R_32F, CUSPARSE_SPMM_ALG_DEFAULT, &need);
    if (s == CUSPARSE_STATUS_SUCCESS && need > g->sp_buf_bytes) {
        cudaStreamSynchronize((cudaStream_t)stream);
        if (g->sp_buf) cudaFree(g->sp_buf);
        g->sp_buf = nullptr;
        g->sp_buf_bytes = 0;
        if (cudaMalloc(&g->sp_buf, need) != cudaSuccess) {
            cudaGetLastError();
            s = CUSPARSE_STATUS_ALLOC_FAILED;
        } else {
            g->sp_buf_bytes = need;
        }
    }
    if (s == CUSPARSE_STATUS_SUCCESS)
        s = cusparseSpMM(h, CUSPARSE_OPERATION_NON_TRANSPOSE, CUSPARSE_OPERATION_NON_TRANSPOSE, &one, mat, mx, &zero,
                         my, CUDA_R_32F, CUSPARSE_SPMM_ALG_DEFAULT, g->sp_buf);
    cusparseDestroyDnMat(mx);
    cusparseDestroyDnMat(my);
    BVG_SP_TRY(s, who);
    return BVG_OK;
}

}  // namespace

extern "C" int bvg_csr_cusparse_Ax(const bvg_csr_graph* g, const float* x, float* y, int32_t k, int64_t ld,
                                   void* stream) {
    if (!g) return fail(BVG_ERR_INVALID_ARG, "bvg_csr_cusparse_Ax: NULL graph");
    return cusparse_product(const_cast<bvg_csr_graph*>(g), false, x, y, k, ld, stream, "bvg_csr_cusparse_Ax");
}

extern "C" int bvg_csr_cusparse_xA(const bvg_csr_graph* g, const float* x, float* y, int32_t k, int64_t ld,
                                   void* stream) {
    if (!g) return fail(BVG_ERR_INVALID_ARG, "bvg_csr_cusparse_xA: NULL graph");
    return cusparse_product(const_cast<bvg_csr_graph*>(g), true, x, y, k, ld, stream, "bvg_csr_cusparse_xA");
}

extern "C" void bvg_free_csr(bvg_csr_graph* g) {
    if (!g) return;
    if (g->sp_mat) cusparseDestroySpMat((cusparseSpMatDescr_t)g->sp_mat);
    if (g->sp_matt) cusparseDestroySpMat((cusparseSpMatDescr_t)g->sp_matt);
    if (g->sp_handle) cusparseDestroy((cusparseHandle_t)g->sp_handle);
    for (void* p : {(void*)g->rp, (void*)g->ci, (void*)g->rpt, (void*)g->cit, (void*)g->hub, (void*)g->hubt,
                    (void*)g->rp32, (void*)g->rpt32, (void*)g->ones, g->sp_buf})
        if (p) cudaFree(p);
    delete g;
}

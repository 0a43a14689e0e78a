// Products on the biclique representation (the second compressed format of
// the paper's final remarks, Sec. 6) on the device.
//
// A x^T follows the passage's steps: c_r = sum_{j in C_r} x_j for every
// biclique (one launch, a lane group per biclique), then y_i = sum of c_r over
// the bicliques whose S holds row i, plus x_j over row i's residual edges
// (a second launch, a lane group per row, gathering; no atomics). x A is the
// transpose: d_r = sum_{i in S_r} x_i, then y_j = sum of d_r over the bicliques
// whose C holds column j, plus x_i over the residual edges into column j.
// Every sum is compensated (two_sum, the errors added in FP32) and rounded
// once: the per-biclique sums into scratch, the gathered sums into y. There
// are only +1 entries, so no sum cancels and the error stays within a few
// units in the last place of the product's own terms.
#include <algorithm>
#include <new>
#include <vector>

#include "device_common.cuh"

using namespace bvg;

struct bvg_biclique_dev {
    int64_t n = 0, m = 0, nb = 0;
    int device = 0;
    // bicliques: members on each side
    uint32_t *s_ptr = nullptr, *s_idx = nullptr, *c_ptr = nullptr, *c_idx = nullptr;
    // gather lists: bicliques per row (S side) and per column (C side);
    // residual edges by row and by column
    uint32_t *row_ptr2 = nullptr, *row_bic = nullptr, *col_ptr2 = nullptr, *col_bic = nullptr;
    uint32_t *r_ptr = nullptr, *r_col = nullptr, *rt_ptr = nullptr, *rt_row = nullptr;
    float* sums = nullptr;  // per-biclique sums, nb x kcap
    int64_t kcap = 0;
    // lists longer than kBicHub entries, summed by a whole CTA each: bicliques
    // by their S and by their C side, rows (bicliques of S + residual edges)
    // and columns (bicliques of C + residual edges)
    uint32_t *hub_s = nullptr, *hub_c = nullptr, *hub_row = nullptr, *hub_col = nullptr;
    int64_t nhub_s = 0, nhub_c = 0, nhub_row = 0, nhub_col = 0;
};


namespace bvg {

// Lists with more entries than this are summed by a whole CTA: one lane
// group walking a hub row of a power-law graph (up to 200,000 residual edges)
// would hold up the whole launch.
constexpr uint32_t kBicHub = 256;

// Lane groups of G = KB / V lanes, one list each: out[l] = sum of
// x[idx[e]] over e in [ptr[l], ptr[l + 1]) (compensated, rounded once).
// Lists longer than kBicHub are left to k_bic_hub.
template <int KB, int V>
__global__ void __launch_bounds__(256) k_bic_sums(const uint32_t* __restrict__ ptr, const uint32_t* __restrict__ idx,
                                                 int64_t lists, const float* __restrict__ x, int64_t ldx,
                                                 float* __restrict__ out, int64_t ldo) {
    constexpr int G = KB / V;
    const int64_t l = (int64_t)blockIdx.x * (256 / G) + threadIdx.x / G;
    const int lane = threadIdx.x % G;
    if (l >= lists) return;
    df acc[V];
#pragma unroll
    for (int v = 0; v < V; v++) acc[v] = df_zero();
    const uint32_t e0 = __ldg(ptr + l), e1 = __ldg(ptr + l + 1);
    if (e1 - e0 > kBicHub) return;
    for (uint32_t e = e0; e < e1; e++) {
        const Vec<V> xv = ldv<V>(x + (int64_t)__ldg(idx + e) * ldx + lane * V);
#pragma unroll
        for (int v = 0; v < V; v++) acc[v] = df_addf(acc[v], xv.v[v]);
    }
    Vec<V> o;
#pragma unroll
    for (int v = 0; v < V; v++) o.v[v] = df_val(acc[v]);
    stv<V>(out + l * ldo + lane * V, o);
}

// One long list per CTA: out[l] = sum of src[idx[e]] over e in
// [ptr[l], ptr[l + 1]) plus, when ptr2 is given, sum of src2[idx2[e]] over
// [ptr2[l], ptr2[l + 1]). Each lane group sums a strided share compensated,
// the groups of a warp combine by a fixed shuffle tree and one thread per
// right-hand side adds the warps in order (deterministic).
template <int KB, int V>
__global__ void __launch_bounds__(256) k_bic_hub(const uint32_t* __restrict__ hubs, const uint32_t* __restrict__ ptr,
                                                const uint32_t* __restrict__ idx, const float* __restrict__ src,
                                                int64_t lds, const uint32_t* __restrict__ ptr2,
                                                const uint32_t* __restrict__ idx2, const float* __restrict__ src2,
                                                int64_t lds2, float* __restrict__ out, int64_t ldo) {
    constexpr int G = KB / V, NGR = 256 / G, NW = 8;
    __shared__ df part[NW][KB];
    const int g = threadIdx.x / G, lane = threadIdx.x % G, lane32 = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t l = __ldg(hubs + blockIdx.x);
    df acc[V];
#pragma unroll
    for (int v = 0; v < V; v++) acc[v] = df_zero();
    const uint32_t e1 = __ldg(ptr + l + 1);
    for (uint32_t e = __ldg(ptr + l) + g; e < e1; e += NGR) {
        const Vec<V> xv = ldv<V>(src + (int64_t)__ldg(idx + e) * lds + lane * V);
#pragma unroll
        for (int v = 0; v < V; v++) acc[v] = df_addf(acc[v], xv.v[v]);
    }
    if (ptr2) {
        const uint32_t f1 = __ldg(ptr2 + l + 1);
        for (uint32_t e = __ldg(ptr2 + l) + g; e < f1; e += NGR) {
            const Vec<V> xv = ldv<V>(src2 + (int64_t)__ldg(idx2 + e) * lds2 + lane * V);
#pragma unroll
            for (int v = 0; v < V; v++) acc[v] = df_addf(acc[v], xv.v[v]);
        }
    }
#pragma unroll
    for (int v = 0; v < V; v++)
        for (int o = G; o < 32; o <<= 1) acc[v] = df_add(acc[v], df_shfl_xor(acc[v], o));
    if (lane32 < G) {
#pragma unroll
        for (int v = 0; v < V; v++) part[warp][lane32 * V + v] = acc[v];
    }
    __syncthreads();
    if (threadIdx.x < KB) {
        df t = df_zero();
        for (int w = 0; w < NW; w++) t = df_add(t, part[w][threadIdx.x]);
        out[l * ldo + threadIdx.x] = df_val(t);
    }
}

// One lane group per output row: y_i = sum of sums[bic] over the row's
// bicliques + sum of x[res] over its residual edges (compensated, rounded
// once).
template <int KB, int V>
__global__ void __launch_bounds__(256) k_bic_gather(const uint32_t* __restrict__ bptr, const uint32_t* __restrict__ bic,
                                                   const float* __restrict__ sums, int64_t lds,
                                                   const uint32_t* __restrict__ rptr, const uint32_t* __restrict__ res,
                                                   const float* __restrict__ x, int64_t ldx, float* __restrict__ y,
                                                   int64_t ldy, int64_t n) {
    constexpr int G = KB / V;
    const int64_t i = (int64_t)blockIdx.x * (256 / G) + threadIdx.x / G;
    const int lane = threadIdx.x % G;
    if (i >= n) return;
    df acc[V];
#pragma unroll
    for (int v = 0; v < V; v++) acc[v] = df_zero();
    const uint32_t b0 = __ldg(bptr + i), b1 = __ldg(bptr + i + 1);
    if ((b1 - b0) + (__ldg(rptr + i + 1) - __ldg(rptr + i)) > kBicHub) return;  // k_bic_hub
    for (uint32_t e = b0; e < b1; e++) {
        const Vec<V> sv = ldv<V>(sums + (int64_t)__ldg(bic + e) * lds + lane * V);
#pragma unroll
        for (int v = 0; v < V; v++) acc[v] = df_addf(acc[v], sv.v[v]);
    }
    const uint32_t r1 = __ldg(rptr + i + 1);
    for (uint32_t e = __ldg(rptr + i); e < r1; e++) {
        const Vec<V> xv = ldv<V>(x + (int64_t)__ldg(res + e) * ldx + lane * V);
#pragma unroll
        for (int v = 0; v < V; v++) acc[v] = df_addf(acc[v], xv.v[v]);
    }
    Vec<V> o;
#pragma unroll
    for (int v = 0; v < V; v++) o.v[v] = df_val(acc[v]);
    stv<V>(y + i * ldy + lane * V, o);
}

template <int KB, int V>
static void launch_bic(const bvg_biclique_dev* d, bool left, const float* x, int64_t ld, float* y,
                       cudaStream_t st) {
    constexpr int G = KB / V, PER = 256 / G;
    const uint32_t* sp = left ? d->s_ptr : d->c_ptr;
    const uint32_t* si = left ? d->s_idx : d->c_idx;
    if (d->nb > 0) {
        const int64_t grid = (d->nb + PER - 1) / PER;
        k_bic_sums<KB, V><<<(unsigned)grid, 256, 0, st>>>(sp, si, d->nb, x, ld, d->sums, KB);
        const int64_t nh = left ? d->nhub_s : d->nhub_c;
        if (nh > 0)
            k_bic_hub<KB, V><<<(unsigned)nh, 256, 0, st>>>(left ? d->hub_s : d->hub_c, sp, si, x, ld, nullptr,
                                                           nullptr, nullptr, 0, d->sums, KB);
    }
    const uint32_t* bp = left ? d->col_ptr2 : d->row_ptr2;
    const uint32_t* bl = left ? d->col_bic : d->row_bic;
    const uint32_t* rp = left ? d->rt_ptr : d->r_ptr;
    const uint32_t* rl = left ? d->rt_row : d->r_col;
    const int64_t grid = (d->n + PER - 1) / PER;
    k_bic_gather<KB, V><<<(unsigned)grid, 256, 0, st>>>(bp, bl, d->sums, KB, rp, rl, x, ld, y, ld, d->n);
    const int64_t nh = left ? d->nhub_col : d->nhub_row;
    if (nh > 0)
        k_bic_hub<KB, V><<<(unsigned)nh, 256, 0, st>>>(left ? d->hub_col : d->hub_row, bp, bl, d->sums, KB, rp, rl,
                                                       x, ld, y, ld);
}

static int bic_product(bvg_biclique_dev* d, bool left, const float* x, float* y, int32_t k, int64_t ld,
                       void* stream, const char* who) {
    if (!d) return fail(BVG_ERR_INVALID_ARG, "%s: NULL handle", who);
    if (k < 1 || ld < k || !x || !y) return fail(BVG_ERR_INVALID_ARG, "%s: bad k/ld or NULL vector", who);
    if ((uintptr_t)x % 4 || (uintptr_t)y % 4) return fail(BVG_ERR_INVALID_ARG, "%s: misaligned vector", who);
    if (x == y) return fail(BVG_ERR_INVALID_ARG, "%s: x and y must not alias", who);
    if (d->n == 0) return BVG_OK;
    cudaStream_t st = (cudaStream_t)stream;
    for (int64_t c0 = 0; c0 < k;) {
        int kb = 32;
        while (kb > k - c0) kb >>= 1;
        if (d->kcap < kb) {
            BVG_CUDA_TRY(cudaStreamSynchronize(st));  // earlier products may still read the old sums
            if (d->sums) cudaFree(d->sums);
            d->sums = nullptr;
            d->kcap = 0;
            if (cudaMalloc(&d->sums, (size_t)std::max<int64_t>(d->nb, 1) * kb * sizeof(float)) != cudaSuccess) {
                cudaGetLastError();
                return fail(BVG_ERR_OOM, "%s: scratch allocation failed", who);
            }
            d->kcap = kb;
        }
        auto ok = [&](int v) {
            if (kb % v || ld % v || c0 % v) return false;
            return (uintptr_t)(x + c0) % (4 * v) == 0 && (uintptr_t)(y + c0) % (4 * v) == 0;
        };
        const int v = (kb >= 4 && ok(4)) ? 4 : ((kb == 2 && ok(2)) ? 2 : 1);
        switch (kb * 8 + v) {
            case 1 * 8 + 1: launch_bic<1, 1>(d, left, x + c0, ld, y + c0, st); break;
            case 2 * 8 + 1: launch_bic<2, 1>(d, left, x + c0, ld, y + c0, st); break;
            case 2 * 8 + 2: launch_bic<2, 2>(d, left, x + c0, ld, y + c0, st); break;
            case 4 * 8 + 1: launch_bic<4, 1>(d, left, x + c0, ld, y + c0, st); break;
            case 4 * 8 + 4: launch_bic<4, 4>(d, left, x + c0, ld, y + c0, st); break;
            case 8 * 8 + 1: launch_bic<8, 1>(d, left, x + c0, ld, y + c0, st); break;
            case 8 * 8 + 4: launch_bic<8, 4>(d, left, x + c0, ld, y + c0, st); break;
            case 16 * 8 + 1: launch_bic<16, 1>(d, left, x + c0, ld, y + c0, st); break;
            case 16 * 8 + 4: launch_bic<16, 4>(d, left, x + c0, ld, y + c0, st); break;
            case 32 * 8 + 1: launch_bic<32, 1>(d, left, x + c0, ld, y + c0, st); break;
            case 32 * 8 + 4: launch_bic<32, 4>(d, left, x + c0, ld, y + c0, st); break;
            default: return fail(BVG_ERR_INVALID_ARG, "%s: no kernel for kb=%d v=%d", who, kb, v);
        }
        c0 += kb;
    }
    BVG_CUDA_TRY(cudaGetLastError());
    return BVG_OK;
}

}  // namespace bvg

extern "C" int bvg_biclique_upload(const bvg_biclique* b, void* stream, bvg_biclique_dev** out) {
    if (!b || !out) return fail(BVG_ERR_INVALID_ARG, "bvg_biclique_upload: NULL argument");
    *out = nullptr;
    const int64_t n = b->n, nb = (int64_t)b->s_ptr.size() - 1;
    const int64_t lim = ((int64_t)1 << 32) - 1;
    if (n >= lim || (int64_t)b->s_idx.size() >= lim || (int64_t)b->c_idx.size() >= lim ||
        (int64_t)b->r_col.size() >= lim)
        return fail(BVG_ERR_UNSUPPORTED, "bvg_biclique_upload: 2^32 list entries or more");
    bvg_biclique_dev* d = new (std::nothrow) bvg_biclique_dev();
    if (!d) return fail(BVG_ERR_OOM, "bvg_biclique_upload: host allocation failed");
    d->n = n;
    d->m = b->m;
    d->nb = nb;
    cudaGetDevice(&d->device);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = BVG_OK;
    try {
        // gather lists (the same counting sorts as bvg_biclique_gather_lists)
        std::vector<int64_t> rp2(n + 1), cp2(n + 1), rtp(n + 1);
        std::vector<int32_t> rb(b->s_idx.size()), cb(b->c_idx.size()), rtr(b->r_col.size());
        if ((rc = bvg_biclique_gather_lists(b, rp2.data(), rb.data(), cp2.data(), cb.data(), rtp.data(), rtr.data())))
            throw rc;
        auto u32 = [](const auto& v) { return std::vector<uint32_t>(v.begin(), v.end()); };
        // the long lists (k_bic_hub)
        std::vector<uint32_t> hs, hc, hr, hcol;
        for (int64_t r = 0; r < nb; r++) {
            if (b->s_ptr[r + 1] - b->s_ptr[r] > kBicHub) hs.push_back((uint32_t)r);
            if (b->c_ptr[r + 1] - b->c_ptr[r] > kBicHub) hc.push_back((uint32_t)r);
        }
        for (int64_t i = 0; i < n; i++) {
            if ((rp2[i + 1] - rp2[i]) + (b->r_ptr[i + 1] - b->r_ptr[i]) > kBicHub) hr.push_back((uint32_t)i);
            if ((cp2[i + 1] - cp2[i]) + (rtp[i + 1] - rtp[i]) > kBicHub) hcol.push_back((uint32_t)i);
        }
        d->nhub_s = (int64_t)hs.size();
        d->nhub_c = (int64_t)hc.size();
        d->nhub_row = (int64_t)hr.size();
        d->nhub_col = (int64_t)hcol.size();
        std::vector<std::vector<uint32_t>> host = {u32(b->s_ptr), u32(b->s_idx), u32(b->c_ptr), u32(b->c_idx),
                                                  u32(rp2),      u32(rb),       u32(cp2),      u32(cb),
                                                  u32(b->r_ptr), u32(b->r_col), u32(rtp),      u32(rtr),
                                                  hs,            hc,            hr,            hcol};
        uint32_t** dst[] = {&d->s_ptr,    &d->s_idx,   &d->c_ptr, &d->c_idx, &d->row_ptr2, &d->row_bic,
                            &d->col_ptr2, &d->col_bic, &d->r_ptr, &d->r_col, &d->rt_ptr,   &d->rt_row,
                            &d->hub_s,    &d->hub_c,   &d->hub_row, &d->hub_col};
        for (size_t t = 0; t < host.size(); t++) {
            const size_t bytes = std::max<size_t>(host[t].size(), 1) * sizeof(uint32_t);
            if (inject_alloc_failure() || cudaMalloc((void**)dst[t], bytes) != cudaSuccess) {
                cudaGetLastError();
                throw (int)BVG_ERR_OOM;
            }
            if (!host[t].empty() &&
                cudaMemcpyAsync(*dst[t], host[t].data(), host[t].size() * sizeof(uint32_t), cudaMemcpyHostToDevice,
                                st) != cudaSuccess) {
                cudaGetLastError();
                throw (int)BVG_ERR_CUDA;
            }
        }
        if (cudaStreamSynchronize(st) != cudaSuccess) {  // the host vectors go out of scope
            cudaGetLastError();
            throw (int)BVG_ERR_CUDA;
        }
    } catch (int code) {
        bvg_free_biclique_dev(d);
        return code == BVG_ERR_OOM ? fail(BVG_ERR_OOM, "bvg_biclique_upload: allocation failed")
                                   : (code == BVG_ERR_CUDA ? fail(BVG_ERR_CUDA, "bvg_biclique_upload: copy failed")
                                                           : code);
    } catch (const std::bad_alloc&) {
        bvg_free_biclique_dev(d);
        return fail(BVG_ERR_OOM, "bvg_biclique_upload: host allocation failed");
    }
    *out = d;
    return BVG_OK;
}

extern "C" int bvg_biclique_spmv_Ax(const bvg_biclique_dev* d, const float* x, float* y, int32_t k, int64_t ld,
                                    void* stream) {
    return bic_product(const_cast<bvg_biclique_dev*>(d), false, x, y, k, ld, stream, "bvg_biclique_spmv_Ax");
}

extern "C" int bvg_biclique_spmv_xA(const bvg_biclique_dev* d, const float* x, float* y, int32_t k, int64_t ld,
                                    void* stream) {
    return bic_product(const_cast<bvg_biclique_dev*>(d), true, x, y, k, ld, stream, "bvg_biclique_spmv_xA");
}

extern "C" void bvg_free_biclique_dev(bvg_biclique_dev* d) {
    if (!d) return;
    for (uint32_t* p : {d->s_ptr, d->s_idx, d->c_ptr, d->c_idx, d->row_ptr2, d->row_bic, d->col_ptr2, d->col_bic,
                        d->r_ptr, d->r_col, d->rt_ptr, d->rt_row, d->hub_s, d->hub_c, d->hub_row, d->hub_col})
        if (p) cudaFree(p);
    if (d->sums) cudaFree(d->sums);
    delete d;
}

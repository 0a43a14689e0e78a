// y = A x^T for one right-hand side in a single kernel (Sec. 4: y_i =
// y_{r_i} + sum_j A'_ij x_j, the row's difference sum added to its
// reference's result, resolved along the reference chains).
//
// A CTA owns kPxT consecutive rows [a, a + kPxT) and also reads the kHalo
// rows before them (the rows their chains reach). In shared memory:
//   1. x of the tile's column window (the columns the entries of rows
//      [a - kHalo, a + kPxT) reference, set per tile at upload; coalesced
//      loads), each row's first work item and reference offset;
//   2. the work items of those rows (every interval member an entry, at most
//      8 entries an item, so that long rows do not hold up their lanes): a
//      thread per item sums +-x over its entries (16-bit words: the column's
//      offset in the window of the tile that owns the row, and a sign);
//   3. each row's difference sum c_i = the sum of its items, then
//      y_i = c_i + c_{r_i} + c_{r_{r_i}} + ... (at most max_chain + 1 terms,
//      never reaching before the halo), added from the row outwards.
// No global scratch, no second launch, no atomics.
//
// Exact path (tiles whose window's x span few enough binades, as in the
// one-vector push): every x an int64 multiple of 2^E, every sum exact, y_i
// the exact A x^T rounded once to FP32. Compensated path (wider ranges,
// non-finite values): double-float sums (an error within a few units in the
// last place of the terms' own magnitudes).
#pragma once

#include "fused.cuh"

namespace bvg {

constexpr int kPxT = 1024;                 // rows per CTA
constexpr int kPxNT = 256;                 // threads per CTA
constexpr int kPxRows = kPxT + kHalo;      // rows a CTA reads
constexpr int kPxW = 1792;                 // most columns in a tile's x window (set at upload)
constexpr int kPxXR = kPxW / kPxNT;        // window columns whose x a thread loads
constexpr int kPxItemCap = 2048;           // most work items of a tile (set at upload)
constexpr int kPxItem = 8;                 // most entries of a work item
constexpr int kPxRPT = (kPxRows + kPxNT - 1) / kPxNT;  // rows whose sums a thread forms
static_assert(kPxRows <= kPxW, "the row sums fit the x array");

struct PxArgs {
    const uint32_t* irow;    // n + 1: row i's first work item
    const uint32_t* istart;  // items + 1: item k's first entry
    const uint16_t* pent;    // per entry: the column's offset in the x window of the tile that owns the row
                             // (bits 0-14), a dropped id (bit 15)
    const uint2* ptile;      // per tile of kPxT rows: first and end column of its x window
    const uint8_t* meta;     // reference offset in bits 0-4 (0: no reference)
    const float* x;
    int64_t ldx;
    float* y;
    int64_t ldy;
    int64_t n;
};

struct PxSmem {
    long long v[kPxW];              // x of the window (integers or floats), then the row sums by row
    long long part[kPxItemCap];     // the items' sums (integers, or (hi, lo) float pairs)
    uint32_t irow[kPxRows + 1];
    uint8_t meta[kPxRows];
    unsigned int emax, emin;
};

__global__ void __launch_bounds__(kPxNT, 6) k_pull_fx(PxArgs pa) {
    __shared__ __align__(16) PxSmem S;
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t n = pa.n;
    const int64_t a = (int64_t)blockIdx.x * kPxT;
    const int64_t hi = a + kPxT < n ? a + kPxT : n;
    const int64_t lo = a > kHalo ? a - kHalo : 0;
    const int nrow = (int)(hi - lo), own0 = (int)(a - lo);
    if (tid == 0) {
        S.emax = 0u;
        S.emin = 0xffffffffu;
    }
    // structure that does not depend on x
    const uint2 win = __ldg(pa.ptile + blockIdx.x);
    const int64_t xw0 = win.x;
    const int X = (int)(win.y - win.x);
    // the halo rows' entries are offsets in the previous tile's window
    const int64_t xp0 = blockIdx.x > 0 ? (int64_t)__ldg(pa.ptile + blockIdx.x - 1).x : xw0;
    const int hoff = (int)(xp0 - xw0);
    for (int r = tid; r <= nrow; r += kPxNT) S.irow[r] = __ldg(pa.irow + lo + r);
    for (int r = tid; r < nrow; r += kPxNT) S.meta[r] = __ldg(pa.meta + lo + r);

    // x of the window and its exponent range (as in the one-vector push)
    float xv[kPxXR];
    uint32_t bmax = 0u, bmin = 0xffffffffu;
#pragma unroll
    for (int i = 0; i < kPxXR; i++) {
        const int c = tid + i * kPxNT;
        xv[i] = c < X ? __ldg(pa.x + (xw0 + c) * pa.ldx) : 0.f;
        const uint32_t b = __float_as_uint(xv[i]) & 0x7fffffffu;
        if (c < X) {
            bmax = max(bmax, b);
            bmin = min(bmin, b ? b : 0xffffffffu);
        }
    }
    bmax = __reduce_max_sync(0xffffffffu, bmax);
    bmin = __reduce_min_sync(0xffffffffu, bmin);
    __syncthreads();  // emax / emin initialised; the rows' items and offsets in place
    if (lane == 0) {
        atomicMax(&S.emax, bmax);
        atomicMin(&S.emin, bmin);
    }
    const uint32_t K0 = S.irow[0], K1 = S.irow[nrow], Ka = S.irow[own0];
    __syncthreads();
    const uint32_t vmax = S.emax >> 23;
    const uint32_t vmin = S.emin == 0xffffffffu ? 255u : max(S.emin >> 23, 1u);
    // headroom: an item adds at most kPxItem values, a row at most the
    // tile's items, a chain at most kMaxChain + 1 rows
    const int hz = 8 + bits_for(kPxItem * (K1 - K0) + 1);
    const int eshift = 38 - hz - (int)vmax;
    const int E = -150 - eshift;
    const bool exact = vmax < 255u && (vmin == 255u || (int)vmin + eshift >= 0);
    if (exact) {
#pragma unroll
        for (int i = 0; i < kPxXR; i++) {
            const int c = tid + i * kPxNT;
            if (c < X) S.v[c] = fx_of(xv[i], E);
        }
    } else {
        float* xs = reinterpret_cast<float*>(S.v);
#pragma unroll
        for (int i = 0; i < kPxXR; i++) {
            const int c = tid + i * kPxNT;
            if (c < X) xs[c] = xv[i];
        }
    }
    __syncthreads();
    // the items: straight-line code over kPxItem predicated entries
    for (uint32_t k = K0 + tid; k < K1; k += kPxNT) {
        const uint32_t e0 = __ldg(pa.istart + k), e1 = __ldg(pa.istart + k + 1);
        const int base = k < Ka ? hoff : 0;
        uint32_t w[kPxItem];
#pragma unroll
        for (int t = 0; t < kPxItem; t++) w[t] = e0 + t < e1 ? (uint32_t)__ldg(pa.pent + e0 + t) : 0u;
        if (exact) {
            long long s = 0;
#pragma unroll
            for (int t = 0; t < kPxItem; t++) {
                if (e0 + t >= e1) break;
                const long long z = S.v[base + (int)(w[t] & 0x7fffu)];
                const long long ng = -(long long)(w[t] >> 15);  // -1: a dropped id
                s += (z ^ ng) - ng;
            }
            S.part[k - K0] = s;
        } else {
            const float* xs = reinterpret_cast<const float*>(S.v);
            df s = df_zero();
#pragma unroll
            for (int t = 0; t < kPxItem; t++) {
                if (e0 + t >= e1) break;
                const float z = xs[base + (int)(w[t] & 0x7fffu)];
                s = df_addf(s, (w[t] >> 15) ? -z : z);
            }
            reinterpret_cast<float2*>(S.part)[k - K0] = make_float2(s.hi, s.lo);
        }
    }
    __syncthreads();
    // each row's sum of its items (in item order), held until every thread
    // has read x, then stored by row in place of x
    long long cs[kPxRPT];
    df cf[kPxRPT];
#pragma unroll
    for (int i = 0; i < kPxRPT; i++) {
        const int r = tid + i * kPxNT;
        cs[i] = 0;
        cf[i] = df_zero();
        if (r >= nrow) continue;
        const uint32_t k0 = S.irow[r] - K0, k1 = S.irow[r + 1] - K0;
        if (exact) {
            for (uint32_t k = k0; k < k1; k++) cs[i] += S.part[k];
        } else {
            const float2* pp = reinterpret_cast<const float2*>(S.part);
            for (uint32_t k = k0; k < k1; k++) cf[i] = df_add(cf[i], {pp[k].x, pp[k].y});
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kPxRPT; i++) {
        const int r = tid + i * kPxNT;
        if (r >= nrow) continue;
        if (exact)
            S.v[r] = cs[i];
        else
            reinterpret_cast<float2*>(S.v)[r] = make_float2(cf[i].hi, cf[i].lo);
    }
    __syncthreads();
    // y_i along the chain, rows in natural order (coalesced stores)
#pragma unroll
    for (int i = 0; i < kPxRPT; i++) {
        const int r = own0 + tid + i * kPxNT;
        if (r >= nrow) continue;
        // the row, then its references (at most kMaxChain, never before the
        // halo): exact in any order; compensated from the row outwards
        float out;
        if (exact) {
            long long s = S.v[r];
            int cur = r;
#pragma unroll
            for (int t = 0; t < kMaxChain; t++) {
                const int off = S.meta[cur] & kMetaOff;
                if (off == 0 || cur - off < 0) break;
                cur -= off;
                s += S.v[cur];
            }
            out = fx_to_float(s, E);
        } else {
            const float2* cc = reinterpret_cast<const float2*>(S.v);
            df s = {cc[r].x, cc[r].y};
            int cur = r;
#pragma unroll
            for (int t = 0; t < kMaxChain; t++) {
                const int off = S.meta[cur] & kMetaOff;
                if (off == 0 || cur - off < 0) break;
                cur -= off;
                s = df_add(s, {cc[cur].x, cc[cur].y});
            }
            out = df_val(s);
        }
        pa.y[(lo + r) * pa.ldy] = out;
    }
}

// Whether the one-vector pull runs as this kernel, and its arguments (api.cu).
bool use_pull_fused(const bvg_dev_graph* g, int kb);
PxArgs pull_fused_args(const bvg_dev_graph* g, const float* x, int64_t ldx, float* y, int64_t ldy);

}  // namespace bvg

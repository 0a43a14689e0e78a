// y = x A for one right-hand side in a single kernel (the push of
// Proposition 1 read for the left product: x A = sum_k z_k a'_k, with z_k the
// sum of x over the rows whose reference chain passes through k).
//
// A CTA owns kFxT consecutive columns [a, a + kFxT) and computes, in shared
// memory, everything its columns need:
//   1. the reference offsets (meta) of a window of rows around the tile, one
//      TMA bulk copy (cp.async.bulk, mbarrier completion), and x of those rows
//      (plain coalesced loads);
//   2. the chain weights z of the window rows;
//   3. the entries of its columns, +-z_k into each column's sums;
//   4. the running interval sum and y_j, rounded once.
// No global scratch, no second launch, no grid-wide synchronisation. Two
// arithmetic paths, chosen per tile (the same choice in every thread):
//
// Exact path (tiles whose x span at most about 20 binades: the rule is
// below). Every value is an int64 multiple of 2^E, E chosen per CTA from the
// largest exponent of the x the tile reads and the number of terms any of its
// sums can hold, so that no sum overflows and every x converts exactly.
//   - chain: every row adds its x into itself and its (at most max_chain)
//     ancestors with shared-memory integer atomics: the pushes of the chain
//     step, in any order, since integer addition is exact and associative;
//   - entries: the tile's event-column entries (points, interval start and
//     end events) dealt evenly over the threads (coalesced), each adding +-z_k
//     into its column's point sum or event sum (integer atomics);
//   - the interval sum: an exact integer prefix of the event sums, each warp
//     starting from the z of the intervals open at its first column (the carry
//     list of its 128 columns);
//   - y_j = P_j + I_j, exact, rounded once to FP32.
// Every result is the exactly rounded sum; an interval that opened and closed
// earlier in the tile leaves nothing behind in the running sum.
//
// Compensated path (tiles whose x span more binades, or hold a non-finite
// value): the chain weights in compensated FP32 (each row's descendants added
// in increasing row order, as the two-kernel push), then each column summed
// over the point columns (every interval member its own entry, no running sum
// across columns): runs of at most kTailItem entries in FP32, joined through
// an error-free two_sum. Errors stay within a few units in the last place of
// the column's own terms.
//
// Entries whose source row lies outside the window (rare on graphs with
// locality; flagged per tile at upload) take z from global memory: x of the
// row and of its descendants (descendant mask). Such tiles first scan their
// entries so that the exponent range covers those rows too.
#pragma once

#include "kernels.cuh"

namespace bvg {

constexpr int kFxT = 1024;                 // columns per CTA (a multiple of kCarryTile)
constexpr int kFxNT = 256;                 // threads per CTA
constexpr int kFxCPT = kFxT / kFxNT;       // consecutive columns per thread: a warp's 128 = one carry tile
constexpr int kFxB = 192;                  // window rows before and after the tile
constexpr int kFxW = kFxT + 2 * kFxB;      // window rows
constexpr int kFxXR = (kFxW + kHalo + kFxNT - 1) / kFxNT;  // rows pushed per thread
constexpr int kFxECap = 3584;              // entries per tile with their column expanded in shared memory
constexpr long long kFxWaitCycles = 4000000000LL;  // bound of an mbarrier wait (about 2 s)
static_assert(kFxCPT * 32 == kCarryTile, "a warp's columns form one carry tile");

struct FxArgs {
    const uint8_t* meta;        // n + 32 bytes (padded for the aligned bulk copy)
    const uint32_t* desc;       // descendant masks
    const uint32_t* colp;       // event columns
    const uint32_t* tent;
    const uint32_t* carry_ptr;
    const uint32_t* carry;
    const uint32_t* pcolp;      // point columns (compensated path)
    const uint32_t* pcent;
    const uint8_t* tile_far;    // per tile of kFxT columns: an entry or carry source lies outside the window
    const float* x;
    int64_t ldx;
    const float* rowscale;      // x_i * rowscale_i (PageRank's 1/outdeg), or NULL
    float* y;
    int64_t ldy;
    int64_t n;
    unsigned int* err;          // set to 1 when a bounded wait ran out
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// One TMA bulk copy global -> shared (16-byte aligned addresses, size a
// multiple of 16), completing on the mbarrier.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Waits for phase `parity` of the mbarrier, at most kFxWaitCycles; false if
// the wait ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > kFxWaitCycles) return false;
    }
}

// x (FP32) as an int64 multiple of 2^E: the 24-bit significand shifted left by
// field + eshift (the exact path guarantees a shift >= 0 for nonzero x).
__device__ __forceinline__ long long fx_of(float v, int eshift) {
    const uint32_t b = __float_as_uint(v);
    const int f = (int)((b >> 23) & 0xffu);
    const uint32_t m = f ? ((b & 0x7fffffu) | 0x800000u) : (b & 0x7fffffu);
    const int sh = (f ? f : 1) + eshift;
    unsigned long long u = m;
    u = sh >= 0 ? (u << sh) : 0ull;
    return (b >> 31) ? -(long long)u : (long long)u;
}

// Exponent field of v (0..255; 255 marks Inf / NaN), and the field that fixes
// the position of its lowest significand bit (1 for subnormals; 255 for
// zero, which converts exactly at any scale).
__device__ __forceinline__ uint32_t expo_of(float v) { return (__float_as_uint(v) >> 23) & 0xffu; }
__device__ __forceinline__ uint32_t low_expo_of(float v) {
    const uint32_t b = __float_as_uint(v) & 0x7fffffffu;
    if (b == 0u) return 255u;
    const uint32_t f = b >> 23;
    return f ? f : 1u;
}

__device__ __forceinline__ long long shfl_xor_ll(long long v, int o) {
    return (long long)__shfl_xor_sync(0xffffffffu, (unsigned long long)v, o);
}
__device__ __forceinline__ long long shfl_up_ll(long long v, int o) {
    return (long long)__shfl_up_sync(0xffffffffu, (unsigned long long)v, o);
}

template <bool COHERENT>
__device__ __forceinline__ float fx_load_x(const FxArgs& fa, int64_t r) {
    float v = COHERENT ? __ldcg(fa.x + r * fa.ldx) : __ldg(fa.x + r * fa.ldx);
    if (fa.rowscale) v = __fmul_rn(v, __ldg(fa.rowscale + r));
    return v;
}

// Exponent range (largest field, smallest low field) of the x a row outside
// the window reads: its own and its descendants'.
template <bool COHERENT>
__device__ __forceinline__ void fx_far_range(const FxArgs& fa, int64_t k, uint32_t& emax, uint32_t& emin) {
    float v = fx_load_x<COHERENT>(fa, k);
    emax = max(emax, expo_of(v));
    emin = min(emin, low_expo_of(v));
    for (uint32_t m = __ldg(fa.desc + k); m; m &= m - 1) {
        v = fx_load_x<COHERENT>(fa, k + __ffs(m));
        emax = max(emax, expo_of(v));
        emin = min(emin, low_expo_of(v));
    }
}

// z_k of a row outside the window, exact path.
template <bool COHERENT>
__device__ __forceinline__ long long fx_far_z(const FxArgs& fa, int64_t k, int eshift) {
    long long v = fx_of(fx_load_x<COHERENT>(fa, k), eshift);
    for (uint32_t m = __ldg(fa.desc + k); m; m &= m - 1) v += fx_of(fx_load_x<COHERENT>(fa, k + __ffs(m)), eshift);
    return v;
}

// z_k of a row outside the window, compensated path: the same additions in
// the same order as the window rows' chain weights.
template <bool COHERENT>
__device__ __forceinline__ float fl_far_z(const FxArgs& fa, int64_t k) {
    df acc = {fx_load_x<COHERENT>(fa, k), 0.f};
    for (uint32_t m = __ldg(fa.desc + k); m; m &= m - 1) acc = df_addf(acc, fx_load_x<COHERENT>(fa, k + __ffs(m)));
    return df_val(acc);
}

// Bits needed for c (ceil(log2(c + 1))).
__device__ __forceinline__ int bits_for(uint32_t c) { return 32 - __clz(c); }

// Shared memory of a tile. The exact path's arrays and the compensated
// path's arrays overlap (a tile takes one path).
struct FxSmem {
    union {
        unsigned long long z[kFxW];     // exact: chain weights
        float zf[kFxW];                 // compensated: chain weights
    } a;
    union {
        unsigned long long P[kFxT];     // exact: point sums
        float x[kFxW + kHalo];          // compensated: x of the window
    } b;
    union {
        unsigned long long D[kFxT];     // exact: event sums
        uint32_t desc[kFxW];            // compensated: descendant masks of the window
    } c;
    uint16_t col[kFxECap];              // exact: the column (in the tile) of each entry
    uint8_t meta[kFxW + kHalo + 48];
    uint64_t bar;
    unsigned int emax, emin, state;
};
static_assert(sizeof(float) * (kFxW + kHalo) <= sizeof(unsigned long long) * kFxT, "x fits the point sums");
static_assert(sizeof(uint32_t) * kFxW <= sizeof(unsigned long long) * kFxT, "masks fit the event sums");

// One tile of the fused product. EPI = 0: store y. EPI = 1: PageRank update
// epilogue (see PrArgs), x = the previous iterate scaled by 1/outdeg.
template <int EPI>
__device__ __forceinline__ void fx_tile(int64_t blk, const FxArgs& fa, const PrArgs& pa, FxSmem& S) {
    constexpr bool COH = EPI == 1;  // x was written by the previous kernel (programmatic dependent launch)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n = fa.n;
    const int64_t a = blk * kFxT;
    const int64_t tend = a + kFxT < n ? a + kFxT : n;
    const int64_t w0 = a > kFxB ? a - kFxB : 0;
    const int64_t w1 = a + kFxT + kFxB < n ? a + kFxT + kFxB : n;
    const int64_t px1 = w1 + kHalo < n ? w1 + kHalo : n;  // rows whose x reaches the window's chain weights
    const int W = (int)(w1 - w0);
    const int64_t m0a = w0 & ~(int64_t)15, m1a = (px1 + 15) & ~(int64_t)15;
    const int moff = (int)(w0 - m0a);

    if (tid == 0) {
        mbar_init(&S.bar, 1);
        S.emax = 0u;
        S.emin = 255u;
        S.state = 0u;
    }
    __syncthreads();
    if (tid == 0) {
        const uint32_t bytes = (uint32_t)(m1a - m0a);
        mbar_expect_tx(&S.bar, bytes);
        bulk_g2s(S.meta, fa.meta + m0a, bytes, &S.bar);
    }
    // structure reads that do not depend on x
    const int64_t c0 = a + (int64_t)tid * kFxCPT;
    uint32_t cp[kFxCPT + 1];
#pragma unroll
    for (int q = 0; q <= kFxCPT; q++) cp[q] = __ldg(fa.colp + (c0 + q < tend ? c0 + q : tend));
    const uint32_t E0 = __ldg(fa.colp + a), E1 = __ldg(fa.colp + tend);
    const bool far = __ldg(fa.tile_far + blk) != 0;
    const int64_t wc = a + (int64_t)warp * kCarryTile;  // this warp's first column
    uint32_t cr0 = 0, cr1 = 0, csrc = 0;
    if (wc < n) {
        cr0 = __ldg(fa.carry_ptr + wc / kCarryTile);
        cr1 = __ldg(fa.carry_ptr + wc / kCarryTile + 1);
        if (cr0 + lane < cr1) csrc = __ldg(fa.carry + cr0 + lane);
    }
    const uint32_t ct0 = __ldg(fa.carry_ptr + a / kCarryTile);
    const uint32_t ct1 = __ldg(fa.carry_ptr + (tend + kCarryTile - 1) / kCarryTile);
    if constexpr (EPI == 1) {
        asm volatile("griddepcontrol.wait;" ::: "memory");  // the previous iterate is complete
        // past convergence or max_iter the update does nothing (the state was
        // written by the previous update; the same value in every thread)
        if (__ldcg(&pa.st->done) || __ldcg(&pa.st->iter) >= __ldcg(&pa.st->max_iter)) {
            if (!mbar_wait(&S.bar, 0)) atomicExch(fa.err, 1u);  // no copy may stay in flight
            return;
        }
    }

    // x of the rows that reach the window, and their exponent range
    float xv[kFxXR];
    uint32_t emax = 0u, emin = 255u;
#pragma unroll
    for (int i = 0; i < kFxXR; i++) {
        const int64_t r = w0 + tid + i * kFxNT;
        xv[i] = r < px1 ? fx_load_x<COH>(fa, r) : 0.f;
        emax = max(emax, expo_of(xv[i]));
        emin = min(emin, low_expo_of(xv[i]));
    }
    if (far) {  // rows outside the window that this tile reads (rare)
        for (uint32_t e = E0 + tid; e < E1; e += kFxNT) {
            const int64_t k = id_of(__ldg(fa.tent + e));
            if (k < w0 || k >= w1) fx_far_range<COH>(fa, k, emax, emin);
        }
        for (uint32_t e = ct0 + tid; e < ct1; e += kFxNT) {
            const int64_t k = __ldg(fa.carry + e);
            if (k < w0 || k >= w1) fx_far_range<COH>(fa, k, emax, emin);
        }
    }
    emax = __reduce_max_sync(0xffffffffu, emax);
    emin = __reduce_min_sync(0xffffffffu, emin);
    if (lane == 0) {
        atomicMax(&S.emax, emax);
        atomicMin(&S.emin, emin);
    }
    if (!mbar_wait(&S.bar, 0)) {
        atomicExch(fa.err, 1u);
        atomicOr(&S.state, 1u);
        mbar_wait(&S.bar, 0);  // once more for the copy in flight
    }
    __syncthreads();
    const uint32_t vmax = S.emax, vmin = S.emin;
    // headroom: a chain weight sums at most kHalo + 1 values, any column or
    // prefix sum at most the tile's entries plus its carry sources
    const int hz = 6 + bits_for((E1 - E0) + (ct1 - ct0) + 1);
    const int eshift = 38 - hz - (int)vmax;  // a significand with exponent field f shifts left by f + eshift
    // exact path: every nonzero x converts without loss, nothing is
    // non-finite; the compensated path otherwise (and after a failed copy,
    // whose outputs are NaN)
    const bool exact = vmax < 255u && (vmin == 255u || (int)vmin + eshift >= 0) && S.state == 0u;
    const bool failed = S.state != 0u;

    float yv[kFxCPT];
    if (exact) {
        for (int i = tid; i < kFxW; i += kFxNT) S.a.z[i] = 0ull;
        for (int i = tid; i < kFxT; i += kFxNT) {
            S.b.P[i] = 0ull;
            S.c.D[i] = 0ull;
        }
        const bool expand = E1 - E0 <= (uint32_t)kFxECap;
        if (expand) {  // the column (in the tile) of every entry
#pragma unroll
            for (int q = 0; q < kFxCPT; q++)
                for (uint32_t e = cp[q]; e < cp[q + 1]; e++) S.col[e - E0] = (uint16_t)(tid * kFxCPT + q);
        }
        __syncthreads();
        // chain step: every row adds its x into itself and its ancestors
#pragma unroll
        for (int i = 0; i < kFxXR; i++) {
            int r = tid + i * kFxNT;  // relative to w0
            if (w0 + r >= px1) break;
            const long long v = fx_of(xv[i], eshift);
            if (v == 0) continue;
            if (r < W) atomicAdd(&S.a.z[r], (unsigned long long)v);
#pragma unroll
            for (int h = 0; h < kMaxChain; h++) {
                const int off = S.meta[r + moff] & 7;
                if (!off) break;
                r -= off;
                if (r < 0) break;  // ancestors below the window are not read
                if (r < W) atomicAdd(&S.a.z[r], (unsigned long long)v);
            }
        }
        __syncthreads();
        auto zfx = [&](int64_t k) -> long long {
            const uint64_t rel = (uint64_t)(k - w0);
            if (rel < (uint64_t)W) return (long long)S.a.z[rel];
            return fx_far_z<COH>(fa, k, eshift);
        };
        // the entries: +-z into the point or the event sum of their column
        if (expand) {
            for (uint32_t e = E0 + tid; e < E1; e += kFxNT) {
                const uint32_t w = __ldg(fa.tent + e);
                long long z = zfx(id_of(w));
                if (w & (1u << kIdBits)) z = -z;  // a dropped id, or an interval that ends here
                unsigned long long* dst = (w & (2u << kIdBits)) ? S.c.D : S.b.P;
                atomicAdd(dst + S.col[e - E0], (unsigned long long)z);
            }
        } else {  // too many entries to expand: each thread its own columns
#pragma unroll
            for (int q = 0; q < kFxCPT; q++) {
                long long p = 0, d = 0;
                for (uint32_t e = cp[q]; e < cp[q + 1]; e++) {
                    const uint32_t w = __ldg(fa.tent + e);
                    long long z = zfx(id_of(w));
                    if (w & (1u << kIdBits)) z = -z;
                    if (w & (2u << kIdBits)) d += z;
                    else p += z;
                }
                S.b.P[tid * kFxCPT + q] = (unsigned long long)p;
                S.c.D[tid * kFxCPT + q] = (unsigned long long)d;
            }
        }
        __syncthreads();
        // running interval sum: this warp's carry, then its columns in order
        long long run = 0;
        if (cr0 + lane < cr1) run = zfx(csrc);
        for (uint32_t e = cr0 + 32 + lane; e < cr1; e += 32) run += zfx(__ldg(fa.carry + e));  // rare: > 32 open
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) run += shfl_xor_ll(run, o);
        long long P[kFxCPT], D[kFxCPT], tot = 0;
#pragma unroll
        for (int q = 0; q < kFxCPT; q++) {
            P[q] = (long long)S.b.P[tid * kFxCPT + q];
            D[q] = (long long)S.c.D[tid * kFxCPT + q];
            tot += D[q];
        }
        long long inc = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = shfl_up_ll(inc, o);
            if (lane >= o) inc += t;
        }
        run += inc - tot;  // the warp's earlier threads
        // 2^E as two normal factors (any E in range is then exact)
        const int E = (int)vmax - 188 + hz;
        const int Ea = E / 2, Eb = E - Ea;
        const float fa_ = __uint_as_float((uint32_t)(Ea + 127) << 23), fb_ = __uint_as_float((uint32_t)(Eb + 127) << 23);
#pragma unroll
        for (int q = 0; q < kFxCPT; q++) {
            run += D[q];
            yv[q] = __fmul_rn(__fmul_rn(__ll2float_rn(P[q] + run), fa_), fb_);
        }
    } else {
        // compensated path: x and the masks of the window into shared memory
#pragma unroll
        for (int i = 0; i < kFxXR; i++) {
            const int r = tid + i * kFxNT;
            if (w0 + r < px1) S.b.x[r] = xv[i];
        }
        for (int r = tid; r < W; r += kFxNT) S.c.desc[r] = __ldg(fa.desc + w0 + r);
        __syncthreads();
        for (int r = tid; r < W; r += kFxNT) {  // chain weights, as the two-kernel push forms them
            const uint32_t m1 = S.c.desc[r], m2 = m1 & (m1 - 1), m3 = m2 & (m2 - 1);
            df acc = {S.b.x[r], 0.f};
            acc = df_addf(acc, m1 ? S.b.x[r + __ffs(m1)] : 0.f);
            acc = df_addf(acc, m2 ? S.b.x[r + __ffs(m2)] : 0.f);
            for (uint32_t mm = m3; mm; mm &= mm - 1) acc = df_addf(acc, S.b.x[r + __ffs(mm)]);
            S.a.zf[r] = df_val(acc);
        }
        __syncthreads();
        auto zfl = [&](int64_t k) -> float {
            const uint64_t rel = (uint64_t)(k - w0);
            if (rel < (uint64_t)W) return S.a.zf[rel];
            return fl_far_z<COH>(fa, k);
        };
#pragma unroll
        for (int q = 0; q < kFxCPT; q++) {
            const int64_t j = c0 + q < tend ? c0 + q : tend;
            const uint32_t pb = __ldg(fa.pcolp + j), pe = __ldg(fa.pcolp + (c0 + q < tend ? j + 1 : j));
            float P = 0.f, Pe = 0.f;
            for (uint32_t e0 = pb; e0 < pe; e0 += kTailItem) {  // runs of kTailItem in FP32, joined exactly
                float sr = 0.f;
                const uint32_t e1 = e0 + kTailItem < pe ? e0 + kTailItem : pe;
                for (uint32_t e = e0; e < e1; e++) {
                    const uint32_t w = __ldg(fa.pcent + e);
                    const float sg = (w >> kIdBits) & 1u ? -1.f : 1.f;
                    sr = __fmaf_rn(sg, zfl(id_of(w)), sr);
                }
                float s_, e_;
                two_sum(P, sr, s_, e_);
                P = s_;
                Pe = __fadd_rn(Pe, e_);
            }
            yv[q] = __fadd_rn(P, Pe);
        }
    }

    float Ssum = 0.f, Rs = 0.f, Dg = 0.f, dl = 0.f;
    if constexpr (EPI == 1) dl = (float)__ldcg(pa.sc_prev + 1);
#pragma unroll
    for (int q = 0; q < kFxCPT; q++) {
        const int64_t j = c0 + q;
        if (failed) yv[q] = __uint_as_float(0x7fc00000u);
        if (j >= tend) continue;
        if constexpr (EPI == 0) {
            fa.y[j * fa.ldy] = yv[q];
        } else {
            const float un = 1.0f / (float)n;
            const float io = __ldg(pa.inv_outdeg + j);
            const float qp = __ldcg(pa.q_prev + j * pa.ldq);
            const float p0j = pa.p0 ? __ldg(pa.p0 + j * pa.ldp0) : un;
            const float gj = pa.dangling_uniform ? un : p0j;
            const float qj = pa.alpha * p0j + (1.0f - pa.alpha) * (yv[q] + dl * gj);
            pa.q_new[j * pa.ldq] = qj;
            Ssum = __fadd_rn(Ssum, qj);
            Rs = __fadd_rn(Rs, fabsf(__fsub_rn(qj, qp)));
            if (io == 0.0f) Dg = __fadd_rn(Dg, qj);
        }
    }
    if constexpr (EPI == 1) {
        df Sd[1] = {{Ssum, 0.f}}, Rd[1] = {{Rs, 0.f}}, Dd[1] = {{Dg, 0.f}};
        pr_block_reduce<1, 1, true>(Sd, Rd, Dd, pa, false);
    }
}

// Whether a graph's one-vector column blocks use this kernel, and its
// arguments for a graph (api.cu).
bool use_fused(const bvg_dev_graph* g, int kb);
FxArgs fused_args(const bvg_dev_graph* g, const float* x, int64_t ldx, const float* rowscale, float* y, int64_t ldy);

template <int EPI>
__global__ void __launch_bounds__(kFxNT) k_push_fx(FxArgs fa, PrArgs pa) {
    __shared__ __align__(16) FxSmem S;
    if constexpr (EPI == 1) asm volatile("griddepcontrol.launch_dependents;");
    fx_tile<EPI>(blockIdx.x, fa, pa, S);
}

}  // namespace bvg

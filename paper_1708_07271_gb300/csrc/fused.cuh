// y = x A for one right-hand side in a single kernel (the push of
// Proposition 1 read for the left product: x A = sum_k z_k a'_k, with z_k the
// sum of x over the rows whose reference chain passes through k).
//
// A CTA owns kFxT consecutive columns [a, a + kFxT) and computes, in shared
// memory, everything its columns need:
//   1. the descendant masks of a window of rows around the tile and the
//      tile's column-major entries (16-bit words: the source row's offset in
//      the window and two flags, built at upload), by two TMA bulk copies
//      (cp.async.bulk, mbarrier completion), and x of the window rows
//      (coalesced loads; the entries' copy is issued once x has arrived);
//   2. the chain weights z of the window rows;
//   3. each thread's 4 columns: +-z_k of their entries into the column's
//      point sum or event sum. On the exact path a warp's 128 columns are
//      dealt to its lanes by entry count (the table lane_cols, built at
//      upload): the longest 32 columns go to slot 0, the next 32 to slot 1,
//      and so on, so that a warp's four column loops run about as long as
//      its four longest columns instead of the longest of its lanes' runs
//      of consecutive columns;
//   4. the running interval sum (in column order, through shared memory) and
//      y_j, rounded once.
// No global scratch, no second launch, no atomics, no grid-wide
// synchronisation. Two arithmetic paths, chosen per tile (the same choice in
// every thread):
//
// Exact path (tiles whose x span at most about 20 binades: the rule is
// below). Every value is an int64 multiple of 2^E, E chosen per CTA from the
// largest exponent of the x the tile reads and the number of terms any of its
// sums can hold, so that no sum overflows and every x converts exactly.
//   - chain: each window row adds the x of its descendants (descendant mask),
//     in integers, so the order does not matter and the sum is exact;
//   - entries: points and interval start / end events of the thread's
//     columns, +-z_k into the column's point or event sum;
//   - the interval sum: an exact integer prefix of the event sums, each warp
//     starting from the z of the intervals open at its first column (the carry
//     list of its 128 columns);
//   - y_j = P_j + I_j, exact, rounded once to FP32 (the integer converted
//     with rounding to nearest even, then scaled by an exact power of two).
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
// Tiles that read a row outside their window (rare on graphs with locality;
// flagged per tile at upload) take the compensated path, where such a row's
// z comes from global memory: x of the row and of its descendants (its
// descendant mask), added in the same order as the window rows'.
#pragma once

#include <cstddef>

#include "kernels.cuh"

namespace bvg {

constexpr int kFxT = 1024;                 // columns per CTA (a multiple of kCarryTile)
constexpr int kFxNT = 256;                 // threads per CTA
constexpr int kFxCPT = kFxT / kFxNT;       // consecutive columns per thread: a warp's 128 = one carry tile
constexpr int kFxW = 1792;                 // most window rows: the span of the rows a tile reads (set at upload)
constexpr int kFxXR = (kFxW + kHalo + kFxNT - 1) / kFxNT;  // window rows whose x a thread loads
constexpr int kFxECap = 7040;              // entries per tile staged in shared memory (more: read from global)
constexpr uint32_t kFxOffMask = 0x3fffu;   // 16-bit entry: the source row's offset in the tile's window
constexpr int kFxDescW = 2 * kFxT > kFxW + 8 ? 2 * kFxT : kFxW + 8;  // mask words; then one int64 per column
constexpr long long kFxWaitCycles = 4000000000LL;  // bound of an mbarrier wait (about 2 s)
static_assert(kFxCPT * 32 == kCarryTile, "a warp's columns form one carry tile");
static_assert(kFxW <= (int)kFxOffMask + 1, "a window offset fits the 16-bit entry");
static_assert(kFxNT == 256 && kFxXR <= 8, "row_order: one byte per row of a 256-row block, at most 8 blocks per window");

struct FxArgs {
    const uint32_t* desc;       // descendant masks, padded by 8 words (aligned bulk copies)
    const uint32_t* colp;       // event columns
    const uint16_t* tent16;     // the event columns' entries as 16-bit words, for tiles not flagged far: the
                                // source row's offset in the tile's row window (bits 0-13), negated (bit 14),
                                // an interval event (bit 15); padded by 8 entries (aligned bulk copies)
    const uint32_t* carry_ptr;
    const uint32_t* carry;
    const uint32_t* pcolp;      // point columns (compensated path)
    const uint32_t* pcent;
    const uint4* tile_win;      // per tile of kFxT columns: (first, end) of its row window, and 1 when a row it
                                // reads lies outside (the rows an entry or open interval comes from span more
                                // than kFxW rows)
    const uint32_t* lane_cols;  // per group of kCarryTile columns, 32 words: lane l's four columns (bytes q =
                                // 0..3, offsets in the group), the group's columns sorted by entry count
                                // (most first) and the q-th 32 given to slot q
    const uint32_t* row_order;  // per 4 aligned blocks of kFxNT rows, kFxNT words: byte (b & 3) of word t is
                                // the row (offset in block b) that thread t takes for the chain weights; each
                                // block's rows sorted by descendant count, most first, the q-th 32 given to
                                // warp (q + b) mod 8
    int64_t row_groups;         // groups of 4 blocks in row_order
    const float* x;
    int64_t ldx;
    const float* rowscale;      // x_i * rowscale_i (PageRank's 1/outdeg), or NULL
    float* y;
    int64_t ldy;
    int64_t n;
    unsigned int* err;          // set to 1 when a bounded wait ran out
    int64_t tile0;              // first column tile of the launch (CTA b takes tile tile0 + b)
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

// 2^s as FP32, -126 <= s <= 127.
__device__ __forceinline__ float pow2f(int s) { return __uint_as_float((uint32_t)(s + 127) << 23); }

// x (FP32) as an int64 multiple of 2^E: x * 2^-E, an integer whenever the
// lowest significand bit of x weighs at least 2^E (the exact path's rule).
// The scaling by powers of two is exact (its result is an integer below
// 2^62, a normal float), and so is the conversion.
__device__ __forceinline__ long long fx_of(float v, int E) {
    const int s = -E;
    const float t = s >= -126 && s <= 127 ? __fmul_rn(v, pow2f(s))
                                          : __fmul_rn(__fmul_rn(v, pow2f(s / 2)), pow2f(s - s / 2));
    return __float2ll_rn(t);
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

// v * 2^E rounded once to FP32: v converted with rounding to nearest (ties
// to even), then scaled by 2^E, exactly unless the result is subnormal (a
// second rounding only then). Scales outside the normal range go in two
// steps, the first exact.
__device__ __forceinline__ float fx_to_float(long long v, int E) {
    const float f = __ll2float_rn(v);
    if (E >= -126 && E <= 127) return __fmul_rn(f, pow2f(E));
    return __fmul_rn(__fmul_rn(f, pow2f(E / 2)), pow2f(E - E / 2));
}

// Shared memory of a tile. The exact path's arrays and the compensated
// path's arrays overlap (a tile takes one path).
struct FxSmem {
    union {
        long long v[kFxW + kHalo];  // exact: x of the window rows as integers, then their chain weights in place
        struct {
            float x[kFxW + kHalo];  // compensated: x of the window rows
            float zf[kFxW];         //   and their chain weights
        } c;
    } a;
    alignas(16) uint32_t desc[kFxDescW];    // descendant masks of the window (16-byte aligned superset); after
                                            // the chain weights, the exact path's per-column event sums
    alignas(16) uint16_t ent[kFxECap + 8];  // the tile's event-column entries (16-byte aligned superset), exact path
    uint64_t bar[2];                // mbarriers: [0] masks, [1] entries
    unsigned int emax, emin, state;
};
static_assert(sizeof(float) * (2 * kFxW + kHalo) <= sizeof(long long) * (kFxW + kHalo), "x and z fit");
static_assert(offsetof(FxSmem, desc) % 16 == 0 && offsetof(FxSmem, ent) % 16 == 0, "bulk-copy targets aligned");
static_assert(kFxDescW * sizeof(uint32_t) >= kFxT * sizeof(long long), "one event sum per column fits the masks");

// One tile of the fused product. EPI = 0: store y. EPI = 1: PageRank update
// epilogue (see PrArgs), x = the previous iterate scaled by 1/outdeg.
template <int EPI>
__device__ __forceinline__ void fx_tile(int64_t blk, const FxArgs& fa, const PrArgs& pa, FxSmem& S) {
    constexpr bool COH = EPI == 1;  // x was written by the previous kernel (programmatic dependent launch)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n = fa.n;
    const int64_t a = blk * kFxT;
    const int64_t tend = a + kFxT < n ? a + kFxT : n;
    const uint4 win = __ldg(fa.tile_win + blk);
    const int64_t w0 = win.x, w1 = win.y;  // the rows the tile reads: [w0, w1), at most kFxW
    const bool far = win.z != 0u;
    const int64_t px1 = w1 + kHalo < n ? w1 + kHalo : n;  // rows whose x reaches the window's chain weights
    const int W = (int)(w1 - w0), PX = (int)(px1 - w0);
    const int64_t d0a = w0 & ~(int64_t)3, d1a = (w1 + 3) & ~(int64_t)3;  // mask copy: 16-byte aligned rows
    const int doff = (int)(w0 - d0a);

    if (tid == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        S.emax = 0u;
        S.emin = 0xffffffffu;
        S.state = 0u;
    }
    __syncthreads();
    // structure reads that do not depend on x
    const uint32_t E0 = __ldg(fa.colp + a), E1 = __ldg(fa.colp + tend);
    const uint32_t e0a = E0 & ~7u, e1a = (E1 + 7u) & ~7u;
    const bool staged = e1a - e0a <= (uint32_t)(kFxECap + 8);
    if (tid == 0) {
        const uint32_t bd = (uint32_t)((d1a - d0a) * 4);
        mbar_expect_tx(&S.bar[0], bd);
        bulk_g2s(S.desc, fa.desc + d0a, bd, &S.bar[0]);
    }
    const int64_t c0 = a + (int64_t)tid * kFxCPT;
    const int64_t wc = a + (int64_t)warp * kCarryTile;  // this warp's first column
    // exact path: slot q of this lane is column wc + byte q of oc (columns
    // balanced over the lanes by entry count); identity: columns c0 + q
    const uint32_t oid = 0x03020100u + 0x04040404u * (uint32_t)lane;
    uint32_t oc = wc < n ? __ldg(fa.lane_cols + (wc / kCarryTile) * 32 + lane) : oid;
    uint32_t cb[kFxCPT], ce[kFxCPT];
#pragma unroll
    for (int q = 0; q < kFxCPT; q++) {
        const int64_t j = wc + ((oc >> (8 * q)) & 0xffu);
        cb[q] = __ldg(fa.colp + (j < tend ? j : tend));
        ce[q] = __ldg(fa.colp + (j + 1 < tend ? j + 1 : tend));
    }
    uint32_t cr0 = 0, cr1 = 0, csrc = 0;
    if (wc < n) {
        cr0 = __ldg(fa.carry_ptr + wc / kCarryTile);
        cr1 = __ldg(fa.carry_ptr + wc / kCarryTile + 1);
        if (cr0 + lane < cr1) csrc = __ldg(fa.carry + cr0 + lane);
    }
    // the chain weights' row order for the window's aligned blocks (at most
    // 8 blocks: 3 words), into L2 now, read after the window's x
    const int64_t b0 = w0 >> 8, g0 = b0 >> 2;
    if (tid < 3 * kFxNT / 32 && g0 + tid / (kFxNT / 32) < fa.row_groups)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(fa.row_order + (g0 + tid / (kFxNT / 32)) * kFxNT + (tid % (kFxNT / 32)) * 32));
    const uint32_t ct0 = __ldg(fa.carry_ptr + a / kCarryTile);
    const uint32_t ct1 = __ldg(fa.carry_ptr + (tend + kCarryTile - 1) / kCarryTile);
    if constexpr (EPI == 1) {
        asm volatile("griddepcontrol.wait;" ::: "memory");  // the previous iterate is complete
        // past convergence or max_iter the update does nothing (the state was
        // written by the previous update; the same value in every thread)
        if (__ldcg(&pa.st->done) || __ldcg(&pa.st->iter) >= __ldcg(&pa.st->max_iter)) {
            const bool ok = mbar_wait(&S.bar[0], 0);  // no copy may stay in flight (the entries' is not issued yet)
            if (!ok) atomicExch(fa.err, 1u);
            return;
        }
    }

    // x of the rows that reach the window, and their exponent range (the
    // largest and smallest nonzero magnitude, as bit patterns: their order is
    // the order of the magnitudes)
    float xv[kFxXR];
    uint32_t bmax = 0u, bmin = 0xffffffffu;
#pragma unroll
    for (int i = 0; i < kFxXR; i++) {
        xv[i] = 0.f;
        const int r = tid + i * kFxNT;
        if (r >= PX) break;
        xv[i] = fx_load_x<COH>(fa, w0 + r);
        const uint32_t b = __float_as_uint(xv[i]) & 0x7fffffffu;
        bmax = max(bmax, b);
        bmin = min(bmin, b ? b : 0xffffffffu);
    }
    bmax = __reduce_max_sync(0xffffffffu, bmax);
    bmin = __reduce_min_sync(0xffffffffu, bmin);
    if (lane == 0) {
        atomicMax(&S.emax, bmax);
        atomicMin(&S.emin, bmin);
    }
    __syncthreads();
    // the tile's entries, once the window's x has arrived: the entry copy
    // lands during the conversion and the chain weights, and the x loads do
    // not queue behind it
    if (tid == 0) {
        const uint32_t be = staged ? (e1a - e0a) * 2u : 0u;
        mbar_expect_tx(&S.bar[1], be);
        if (be) bulk_g2s(S.ent, fa.tent16 + e0a, be, &S.bar[1]);
    }
    // exponent fields: the largest (255: a non-finite value), and the one of
    // the lowest significand bit of the smallest nonzero magnitude (255: no
    // nonzero value)
    const uint32_t vmax = S.emax >> 23;
    const uint32_t vmin = S.emin == 0xffffffffu ? 255u : max(S.emin >> 23, 1u);
    // headroom: a chain weight sums at most kHalo + 1 values, any column or
    // prefix sum at most the tile's entries plus its carry sources
    const int hz = 6 + bits_for((E1 - E0) + (ct1 - ct0) + 1);
    const int eshift = 38 - hz - (int)vmax;  // a significand with exponent field f shifts left by f + eshift
    const int E = -150 - eshift;             // the integers count units of 2^E
    // exact path: every source row lies in the window, every nonzero x
    // converts without loss and nothing is non-finite; the compensated path
    // otherwise
    const bool exact = !far && vmax < 255u && (vmin == 255u || (int)vmin + eshift >= 0);

    float yv[kFxCPT];
    if (exact) {
#pragma unroll
        for (int i = 0; i < kFxXR; i++) {
            const int r = tid + i * kFxNT;
            if (r >= PX) break;
            S.a.v[r] = fx_of(xv[i], E);
        }
        if (!mbar_wait(&S.bar[0], 0)) {
            atomicExch(fa.err, 1u);
            atomicOr(&S.state, 1u);
            mbar_wait(&S.bar[0], 0);  // once more for the copy in flight
        }
        __syncthreads();
        // chain weights: each window row adds the x of its descendants
        // (exact, in any order), held until every row has read, then stored
        // in place. Rows go by aligned blocks of kFxNT in the row_order
        // permutation, so that a warp's 32 rows have similar descendant
        // counts (a warp's loop runs as long as its longest mask).
        uint32_t ow[3];
#pragma unroll
        for (int k = 0; k < 3; k++) ow[k] = g0 + k < fa.row_groups ? __ldg(fa.row_order + (g0 + k) * kFxNT + tid) : 0u;
        const int nb = W > 0 ? (int)(((w1 - 1) >> 8) - b0 + 1) : 0;
        // the window's 8 row-order bytes (blocks b0 .. b0 + 7) lined up in two words
        const int s0 = (int)(b0 & 3);
        const uint32_t u0 = __funnelshift_r(ow[0], ow[1], 8 * s0), u1 = __funnelshift_r(ow[1], ow[2], 8 * s0);
        const int rb = (int)((b0 << 8) - w0);  // block b0's first row in the window (-255 .. 0)
        auto row_of = [&](int i) -> int {     // window row of this thread in block b0 + i (outside: >= W)
            return rb + (i << 8) + (int)(((i < 4 ? u0 : u1) >> (8 * (i & 3))) & 0xffu);
        };
        long long zr[kFxXR];
#pragma unroll
        for (int i = 0; i < kFxXR; i++) {
            if (i >= nb) break;
            const int r = row_of(i);
            zr[i] = 0;
            if ((unsigned)r >= (unsigned)W) continue;
            long long z = S.a.v[r];
            for (uint32_t m = S.desc[r + doff]; m; m &= m - 1) z += S.a.v[r + __ffs(m)];
            zr[i] = z;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kFxXR; i++) {
            if (i >= nb) break;
            const int r = row_of(i);
            if ((unsigned)r < (unsigned)W) S.a.v[r] = zr[i];
        }
        if (!mbar_wait(&S.bar[1], 0)) {
            atomicExch(fa.err, 1u);
            atomicOr(&S.state, 1u);
            mbar_wait(&S.bar[1], 0);
        }
        __syncthreads();
        if (S.state != 0u)  // a copy ran out of time: read no staged entry (the outputs are NaN)
#pragma unroll
            for (int q = 0; q < kFxCPT; q++) ce[q] = cb[q];
        // (the tile reads no row outside its window: z of any source row is
        // in shared memory)
        const long long* zv = S.a.v - w0;
        // this lane's columns (slot q: column wc + byte q of oc): the sum of
        // all entries A_q = P_q + D_q, and the event sum D_q into shared
        // memory at the column's place (the masks are no longer read);
        // y_j = P_j + I_j = A_j + I_{j-1}. +-z of an entry's source row into
        // the point or the event sum.
        long long* Ds = reinterpret_cast<long long*>(S.desc) + warp * kCarryTile;
        long long A[kFxCPT];
        auto column = [&](auto&& word, int q) {
            long long a = 0, d = 0;
            for (uint32_t e = cb[q]; e < ce[q]; e++) {  // branch-free: the lanes' loops differ in length only
                const uint32_t w = word(e);
                long long z = S.a.v[w & kFxOffMask];
                const long long ng = (int)(w << 17) >> 31;  // -1: a dropped id, or an interval ending here
                z = (z ^ ng) - ng;
                a += z;
                d += z & (long long)((int)(w << 16) >> 31);  // an interval start or end event
            }
            A[q] = a;
            Ds[(oc >> (8 * q)) & 0xffu] = d;
        };
        if (staged) {
            const uint16_t* ent = S.ent - e0a;
#pragma unroll
            for (int q = 0; q < kFxCPT; q++) column([&](uint32_t e) { return (uint32_t)ent[e]; }, q);
        } else {
#pragma unroll
            for (int q = 0; q < kFxCPT; q++) column([&](uint32_t e) { return (uint32_t)__ldg(fa.tent16 + e); }, q);
        }
        // running interval sum, in column order: this warp's carry, then its
        // columns in order; each column's running sum goes back to the lane
        // holding the column
        __syncwarp();
        long long dq[kFxCPT], tot = 0;
#pragma unroll
        for (int q = 0; q < kFxCPT; q++) {
            dq[q] = Ds[lane * kFxCPT + q];
            tot += dq[q];
        }
        long long run = 0;
        if (cr0 + lane < cr1) run = zv[csrc];
        for (uint32_t e = cr0 + 32 + lane; e < cr1; e += 32) run += zv[__ldg(fa.carry + e)];  // rare: > 32 open
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) run += shfl_xor_ll(run, o);
        long long inc = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = shfl_up_ll(inc, o);
            if (lane >= o) inc += t;
        }
        run += inc - tot;  // the warp's earlier lanes
#pragma unroll
        for (int q = 0; q < kFxCPT; q++) {
            Ds[lane * kFxCPT + q] = run;  // the intervals open before the column
            run += dq[q];
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < kFxCPT; q++) yv[q] = fx_to_float(A[q] + Ds[(oc >> (8 * q)) & 0xffu], E);
    } else {
        oc = oid;  // the compensated path keeps columns c0 + q
        // compensated path: x of the window into shared memory
#pragma unroll
        for (int i = 0; i < kFxXR; i++) {
            const int r = tid + i * kFxNT;
            if (r < PX) S.a.c.x[r] = xv[i];
        }
        if (!mbar_wait(&S.bar[0], 0) || !mbar_wait(&S.bar[1], 0)) {
            atomicExch(fa.err, 1u);
            atomicOr(&S.state, 1u);
            mbar_wait(&S.bar[0], 0);
            mbar_wait(&S.bar[1], 0);
        }
        __syncthreads();
        for (int r = tid; r < W; r += kFxNT) {  // chain weights, as the two-kernel push forms them
            const uint32_t m1 = S.desc[r + doff], m2 = m1 & (m1 - 1), m3 = m2 & (m2 - 1);
            df acc = {S.a.c.x[r], 0.f};
            acc = df_addf(acc, m1 ? S.a.c.x[r + __ffs(m1)] : 0.f);
            acc = df_addf(acc, m2 ? S.a.c.x[r + __ffs(m2)] : 0.f);
            for (uint32_t mm = m3; mm; mm &= mm - 1) acc = df_addf(acc, S.a.c.x[r + __ffs(mm)]);
            S.a.c.zf[r] = df_val(acc);
        }
        __syncthreads();
        auto zfl = [&](int64_t k) -> float {
            const uint64_t rel = (uint64_t)(k - w0);
            if (rel < (uint64_t)W) return S.a.c.zf[rel];
            return fl_far_z<COH>(fa, k);
        };
#pragma unroll
        for (int q = 0; q < kFxCPT; q++) {
            const int64_t j = c0 + q < tend ? c0 + q : tend;
            const uint32_t pb = __ldg(fa.pcolp + j), pe = __ldg(fa.pcolp + (c0 + q < tend ? j + 1 : j));
            float P = 0.f, Pe = 0.f;
            for (uint32_t e0 = pb; e0 < pe; e0 += kTailItem) {  // runs of kTailItem in FP32, joined exactly
                uint32_t w4[kTailItem];
#pragma unroll
                for (int t = 0; t < kTailItem; t++) w4[t] = e0 + t < pe ? __ldg(fa.pcent + e0 + t) : 0u;
                float sr = 0.f;
#pragma unroll
                for (int t = 0; t < kTailItem; t++) {
                    if (e0 + t >= pe) break;
                    const float sg = (w4[t] >> kIdBits) & 1u ? -1.f : 1.f;
                    sr = __fmaf_rn(sg, zfl(id_of(w4[t])), sr);
                }
                float s_, e_;
                two_sum(P, sr, s_, e_);
                P = s_;
                Pe = __fadd_rn(Pe, e_);
            }
            yv[q] = __fadd_rn(P, Pe);
        }
    }
    const bool failed = S.state != 0u;  // a copy ran out of time: NaN outputs

    float Ssum = 0.f, Rs = 0.f, Dg = 0.f, dl = 0.f;
    const float un = EPI == 1 ? 1.0f / (float)n : 0.0f;
    if constexpr (EPI == 1) dl = sc_dangling_f32(pa.sc_prev, 0);
#pragma unroll
    for (int q = 0; q < kFxCPT; q++) {
        const int64_t j = wc + ((oc >> (8 * q)) & 0xffu);
        if (failed) yv[q] = __uint_as_float(0x7fc00000u);
        if (j >= tend) continue;
        if constexpr (EPI == 0) {
            fa.y[j * fa.ldy] = yv[q];
        } else {
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
__global__ void __launch_bounds__(kFxNT, 6) k_push_fx(FxArgs fa, PrArgs pa) {
    __shared__ __align__(16) FxSmem S;
    if constexpr (EPI == 1) asm volatile("griddepcontrol.launch_dependents;");
    fx_tile<EPI>(fa.tile0 + blockIdx.x, fa, pa, S);
}

}  // namespace bvg

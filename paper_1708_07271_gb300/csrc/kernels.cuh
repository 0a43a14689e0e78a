// Kernels of the BV-delta products. Everything here is templated on
//   KB : right-hand sides handled by one launch (1, 2, 4, 8, 16, 32)
//   V  : floats per vector access (1, 2 or 4; KB % V == 0)
// A group of G = KB / V consecutive lanes owns one row (or column); lane l of
// the group owns right-hand sides [l*V, l*V + V).
#pragma once

#include "device_common.cuh"

namespace bvg {

struct PrState {
    int done;      // converged (or non-finite): later kernels return at once
    int numeric;   // a non-finite sum was seen
    int iter;      // completed updates
    int max_iter;
    double tol;
};

// The scalars of an update: 3 x 32 doubles, then 32 floats (the dangling
// mass rounded once, read by every thread of the next update's epilogue).
constexpr int kScDoubles = 3 * 32;
__host__ __device__ constexpr size_t sc_bytes() { return kScDoubles * sizeof(double) + 32 * sizeof(float); }
__device__ __forceinline__ float sc_dangling_f32(const double* sc, int c) {
    return __ldcg(reinterpret_cast<const float*>(sc + kScDoubles) + c);
}

struct PrArgs {
    const float* p0;           // teleport vectors (n x k, ld ldp0) or NULL: seed, else uniform 1/n
    int64_t ldp0;
    const int64_t* seed;       // with p0 NULL: k nodes, teleport vector c = e_seed[c] (one-hot), or NULL
    const float* inv_outdeg;   // 0 marks a row without successors
    const float* q_prev;       // previous iterate, unnormalised (n x k, ld ldq)
    float* q_new;
    float* x_new;              // q_new / outdeg (the next update's input), or NULL
    int64_t ldq;
    const double* sc_prev;     // [3][k]: 1/S, dangling mass, resid (of the previous update), then the
                               // dangling mass rounded to FP32 (kScDanglingF32, k floats)
    double* sc_new;
    PrState* st;
    double* partial;           // [grid][3][KB]
    unsigned int* counter;     // CTAs groups finished (last-group reduction)
    double* gpartial;          // [groups][3][KB]
    unsigned int* gcounter;    // per group of kPrGroup CTAs: CTAs finished
    unsigned int* tile_counter;  // the update gather's next tile (reset by the grid reduction's last CTA
                                 // and by k_pr_init)
    float alpha;
    int dangling_uniform;
    int k;                     // right-hand sides of the solve (== KB)
};


// ---------------------------------------------------------------------------
// Prefix of x (for interval sums of the pull): P(j) = sum_{t < j} x_t, kept
// blocked and compensated: L[j] (hi, lo) is the exclusive prefix inside a
// block of PrefixShape::PB rows, B[b] (hi, lo) the prefix of the block
// starts; P(j) = B[j / PB] + L[j], j = 0..n. An interval sum is then
// P(s + len) - P(s), two differences of compensated values.
// ---------------------------------------------------------------------------
template <int KB, int V>
struct PrefixShape {
    static constexpr int G = KB / V, NG = 256 / G, RPT = 8, PB = NG * RPT;
};

template <int KB, int V>
__global__ void __launch_bounds__(256) k_prefix_local(const float* __restrict__ x, int64_t ldx, float* __restrict__ lhi,
                                                      float* __restrict__ llo, float* __restrict__ bhi,
                                                      float* __restrict__ blo, int64_t n) {
    using Sh = PrefixShape<KB, V>;
    constexpr int G = Sh::G, RPT = Sh::RPT, PB = Sh::PB;
    __shared__ df wtot_s[8][KB];
    const int g = threadIdx.x / G, lane = threadIdx.x % G;
    const int lane32 = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t b0 = (int64_t)blockIdx.x * PB, r0 = b0 + (int64_t)g * RPT;
    df tot[V];
#pragma unroll
    for (int v = 0; v < V; v++) tot[v] = df_zero();
    float xv[RPT][V];
#pragma unroll
    for (int i = 0; i < RPT; i++) {
        Vec<V> t;
#pragma unroll
        for (int v = 0; v < V; v++) t.v[v] = 0.f;
        if (r0 + i < n) t = ldv<V>(x + (r0 + i) * ldx + lane * V);
#pragma unroll
        for (int v = 0; v < V; v++) {
            xv[i][v] = t.v[v];
            tot[v] = df_addf(tot[v], t.v[v]);
        }
    }
    df inc[V], ex[V];
#pragma unroll
    for (int v = 0; v < V; v++) inc[v] = tot[v];
#pragma unroll
    for (int d = G; d < 32; d <<= 1)
#pragma unroll
        for (int v = 0; v < V; v++) {
            df o = df_shfl_up(inc[v], d);
            if (lane32 >= d) inc[v] = df_add_rn(o, inc[v]);
        }
#pragma unroll
    for (int v = 0; v < V; v++) {
        df o = df_shfl_up(inc[v], G);
        ex[v] = lane32 >= G ? o : df_zero();
    }
    if (lane32 >= 32 - G)
#pragma unroll
        for (int v = 0; v < V; v++) wtot_s[warp][lane * V + v] = inc[v];
    __syncthreads();
    df run[V];
#pragma unroll
    for (int v = 0; v < V; v++) {
        df r = df_zero();
        for (int w = 0; w < warp; w++) r = df_add_rn(r, wtot_s[w][lane * V + v]);
        run[v] = df_add_rn(r, ex[v]);
    }
#pragma unroll
    for (int i = 0; i < RPT; i++) {
        if (r0 + i <= n) {
            Vec<V> h, l;
#pragma unroll
            for (int v = 0; v < V; v++) {
                h.v[v] = run[v].hi;
                l.v[v] = run[v].lo;
            }
            stv<V>(lhi + (r0 + i) * KB + lane * V, h);
            stv<V>(llo + (r0 + i) * KB + lane * V, l);
        }
#pragma unroll
        for (int v = 0; v < V; v++) run[v] = df_addf(run[v], xv[i][v]);
    }
    if (threadIdx.x >= 256 - G) {  // the last group holds the block total
#pragma unroll
        for (int v = 0; v < V; v++) {
            bhi[(int64_t)blockIdx.x * KB + lane * V + v] = run[v].hi;
            blo[(int64_t)blockIdx.x * KB + lane * V + v] = run[v].lo;
        }
    }
}

// Exclusive prefix over the nb block totals (one CTA), in place: B[b].
template <int KB>
__global__ void __launch_bounds__(256) k_prefix_blocks(float* __restrict__ bhi, float* __restrict__ blo, int nb) {
    __shared__ df wtot_s[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int per = (nb + 255) / 256, b0 = threadIdx.x * per;
    for (int c = 0; c < KB; c++) {
        df t = df_zero();
        for (int b = b0; b < b0 + per && b < nb; b++) t = df_add_rn(t, {bhi[(int64_t)b * KB + c], blo[(int64_t)b * KB + c]});
        df inc = t;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            df o = df_shfl_up(inc, d);
            if (lane >= d) inc = df_add_rn(o, inc);
        }
        df o = df_shfl_up(inc, 1);
        const df ex = lane >= 1 ? o : df_zero();
        if (lane == 31) wtot_s[warp] = inc;
        __syncthreads();
        df r = df_zero();
        for (int w = 0; w < warp; w++) r = df_add_rn(r, wtot_s[w]);
        r = df_add_rn(r, ex);
        for (int b = b0; b < b0 + per && b < nb; b++) {
            const df cur = {bhi[(int64_t)b * KB + c], blo[(int64_t)b * KB + c]};
            bhi[(int64_t)b * KB + c] = r.hi;
            blo[(int64_t)b * KB + c] = r.lo;
            r = df_add_rn(r, cur);
        }
        __syncthreads();
    }
}

struct PrefixArgs {
    const float* lhi;  // (n+1) x KB
    const float* llo;
    const float* bhi;  // nb x KB (block starts)
    const float* blo;
    int block;         // PB, rows per prefix block
    int min_len;       // intervals at least this long use the prefix
};

// ---------------------------------------------------------------------------
// Pull: y = A x^T (Sec. 4): y_i = y_{r_i} + sum_j A'_ij x_j, in two kernels.
// The row sums c_i = sum_j A'_ij x_j are cut into work items of at most W
// entries (dropped ids subtract, residual ids and the members of intervals
// shorter than a threshold add; the rows of A' differ widely in length, so the
// items, not the rows, are the unit of parallel work):
//   k_pull_items: one item per group of G = KB/V lanes, W straight-line
//     predicated slots (the same instructions for every item), its
//     compensated partial sum rounded once to FP32 and written out (an error
//     of at most u of the item's magnitudes; 4 bytes per item and right-hand
//     side instead of 8);
//   k_pull_rows: a CTA owns rows [a, a + tile); it sums the partials of its
//     rows and of the kHalo rows before them (plus their kept intervals,
//     from the prefix of x or member by member) into shared memory, then
//     resolves each owned row's chain y_i = c_i + c_{r_i} + c_{r_{r_i}} + ...
//     (at most max_chain links, never leaving the kHalo rows), added from the
//     root outwards: the association of the sequential algorithm.
// ---------------------------------------------------------------------------
template <int KB, int V>
__device__ __forceinline__ void pull_interval_prefix(df (&acc)[V], uint32_t s0, uint32_t len, int lane,
                                                     const PrefixArgs& pf) {
    const uint32_t e0 = s0 + len;
    const int64_t bs = s0 / pf.block, be = e0 / pf.block;
    Vec<V> lsh = ldv<V>(pf.lhi + (int64_t)s0 * KB + lane * V), lsl = ldv<V>(pf.llo + (int64_t)s0 * KB + lane * V);
    Vec<V> leh = ldv<V>(pf.lhi + (int64_t)e0 * KB + lane * V), lel = ldv<V>(pf.llo + (int64_t)e0 * KB + lane * V);
    Vec<V> bsh = ldv<V>(pf.bhi + bs * KB + lane * V), bsl = ldv<V>(pf.blo + bs * KB + lane * V);
    Vec<V> beh = ldv<V>(pf.bhi + be * KB + lane * V), bel = ldv<V>(pf.blo + be * KB + lane * V);
#pragma unroll
    for (int v = 0; v < V; v++) {
        const df dB = df_add_rn({beh.v[v], bel.v[v]}, df_neg({bsh.v[v], bsl.v[v]}));
        const df dL = df_add_rn({leh.v[v], lel.v[v]}, df_neg({lsh.v[v], lsl.v[v]}));
        acc[v] = df_add_rn(acc[v], df_add_rn(dB, dL));
    }
}

template <int KB, int V, int W>
__global__ void __launch_bounds__(256) k_pull_items(const uint32_t* __restrict__ pent,
                                                    const uint32_t* __restrict__ istart, int64_t nitems,
                                                    const float* __restrict__ x, int64_t ldx,
                                                    float* __restrict__ part) {
    constexpr int G = KB / V;
    asm volatile("griddepcontrol.launch_dependents;");
    const int64_t k = (int64_t)blockIdx.x * (256 / G) + threadIdx.x / G;
    const int lane = threadIdx.x % G;
    if (k >= nitems) return;
    const uint32_t e0 = __ldg(istart + k), e1 = __ldg(istart + k + 1);
    uint32_t w[W];
#pragma unroll
    for (int t = 0; t < W; t++) w[t] = e0 + t < e1 ? __ldg(pent + e0 + t) : 0u;
    Vec<V> xv[W];
#pragma unroll
    for (int t = 0; t < W; t++) {
#pragma unroll
        for (int v = 0; v < V; v++) xv[t].v[v] = 0.f;
        if (e0 + t < e1) xv[t] = ldv<V>(x + (int64_t)(w[t] & 0x7fffffffu) * ldx + lane * V);
    }
    df acc[V];
#pragma unroll
    for (int v = 0; v < V; v++) acc[v] = df_zero();
#pragma unroll
    for (int t = 0; t < W; t++)
#pragma unroll
        for (int v = 0; v < V; v++) acc[v] = df_addf(acc[v], (w[t] >> 31) ? -xv[t].v[v] : xv[t].v[v]);
    Vec<V> pv;
#pragma unroll
    for (int v = 0; v < V; v++) pv.v[v] = df_val(acc[v]);  // rounded once
    stv<V>(part + k * KB + lane * V, pv);
}

// Adds to acc the items' partial sums k0, k0 + step, ... < k1.
template <int KB, int V>
__device__ __forceinline__ void pull_row_entries(df (&acc)[V], uint32_t k0, uint32_t k1, uint32_t step,
                                                 const float* part, int lane) {
    for (uint32_t k = k0; k < k1; k += step) {
        const Vec<V> p = ldv_cg<V>(part + (int64_t)k * KB + lane * V);
#pragma unroll
        for (int v = 0; v < V; v++) acc[v] = df_addf(acc[v], p.v[v]);
    }
}

// Adds to acc the kept (long) intervals of row i: from the prefix of x, or
// member by member.
template <int KB, int V>
__device__ __forceinline__ void pull_row_intervals(df (&acc)[V], int64_t i, const uint32_t* __restrict__ lrow,
                                                   const uint32_t* __restrict__ lint, const float* __restrict__ x,
                                                   int64_t ldx, int lane, const PrefixArgs& pf) {
    const uint32_t l0 = __ldg(lrow + i), l1 = __ldg(lrow + i + 1);
    for (uint32_t q = l0; q < l1; q++) {  // kept (long) intervals
        const uint32_t s0 = __ldg(lint + 2 * q), len = __ldg(lint + 2 * q + 1);
        if (pf.lhi) {
            pull_interval_prefix<KB, V>(acc, s0, len, lane, pf);
        } else {
            for (uint32_t t = 0; t < len; t++) {
                Vec<V> xv = ldv<V>(x + (int64_t)(s0 + t) * ldx + lane * V);
#pragma unroll
                for (int v = 0; v < V; v++) acc[v] = df_addf(acc[v], xv.v[v]);
            }
        }
    }
}

// Row sum of row i: its items' partial sums [k0, k1), then its kept intervals.
template <int KB, int V>
__device__ __forceinline__ void pull_row_sum(df (&acc)[V], int64_t i, uint32_t k0, uint32_t k1, const float* part,
                                             const uint32_t* __restrict__ lrow, const uint32_t* __restrict__ lint,
                                             const float* __restrict__ x, int64_t ldx, int lane,
                                             const PrefixArgs& pf) {
#pragma unroll
    for (int v = 0; v < V; v++) acc[v] = df_zero();
    pull_row_entries<KB, V>(acc, k0, k1, 1, part, lane);
    pull_row_intervals<KB, V>(acc, i, lrow, lint, x, ldx, lane, pf);
}

// The reference chain of tile row r (indices into the tile's c): r, r's
// reference, ..., at most kMaxChain links, never leaving the kHalo rows.
__device__ __forceinline__ int pull_chain_of(const uint8_t* __restrict__ meta, int64_t lo, int r,
                                             int (&idx)[kMaxChain + 1]) {
    int len = 0, cur = r;
    idx[len++] = cur;
    for (int t = 0; t < kMaxChain; t++) {
        const int off = __ldg(meta + lo + cur) & kMetaOff;
        if (off == 0 || cur - off < 0) break;
        cur -= off;
        idx[len++] = cur;
    }
    return len;
}

// Rows of the row pass with more items than this are summed by the whole CTA
// after the per-group loop, so a hub row (power-law out-degree) does not
// leave one lane group walking it alone.
constexpr uint32_t kPullLongItems = 32;
// Largest row tile of the row pass (rows per CTA, plus the halo).
constexpr int kPullMaxTile = 2048;

template <int KB, int V>
__global__ void __launch_bounds__(256) k_pull_rows(const uint8_t* __restrict__ meta, const uint32_t* __restrict__ irow,
                                                   const float* part, const uint32_t* __restrict__ lrow,
                                                   const uint32_t* __restrict__ lint, const float* __restrict__ x,
                                                   int64_t ldx, float* __restrict__ y, int64_t ldy, int64_t n,
                                                   int tile, PrefixArgs pf) {
    constexpr int G = KB / V;
    // rows per group whose structure is read before the wait (one-lane groups;
    // for wider groups the extra registers cost more than the overlap gains)
    constexpr int PF = G == 1 ? 2 : 0;
    constexpr int PFA = PF > 0 ? PF : 1;
    extern __shared__ float4 smem_pull[];
    // [(tile + kHalo) * KB] row sums, each compensated and then rounded once
    // to FP32 (half the shared memory of keeping them compensated, so twice
    // the resident CTAs for wide column blocks); the chains add them
    // compensated
    float* c = reinterpret_cast<float*>(smem_pull);
    const int NG = blockDim.x / G;
    const int g = threadIdx.x / G, lane = threadIdx.x % G;
    const int64_t a = (int64_t)blockIdx.x * tile;
    const int64_t lo = a > kHalo ? a - kHalo : 0;
    const int64_t hi = a + tile < n ? a + tile : n;
    const int cnt = (int)(hi - lo);
    const int own0 = (int)(a - lo);

    // structure first: it does not depend on the item pass, which may still be
    // running (programmatic dependent launch). The item ranges of the group's
    // first PF rows and the chains of the first PF rows it outputs.
    uint32_t kr[PFA][2];
    int idx[PFA][kMaxChain + 1], clen[PFA];
#pragma unroll
    for (int j = 0; j < PF; j++) {
        const int r = g + j * NG;
        kr[j][0] = r < cnt ? __ldg(irow + lo + r) : 0u;
        kr[j][1] = r < cnt ? __ldg(irow + lo + r + 1) : 0u;
        const int ro = own0 + g + j * NG;
        clen[j] = ro < cnt ? pull_chain_of(meta, lo, ro, idx[j]) : 0;
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");  // the items' partial sums are ready
    constexpr uint32_t kLong = kPullLongItems;
    bool met_long = false;  // this thread's group left a long row for the whole CTA

    auto row_range = [&](int r, uint32_t& k0, uint32_t& k1) {
        k0 = __ldg(irow + lo + r);
        k1 = __ldg(irow + lo + r + 1);
    };
    auto group_row = [&](int r, uint32_t k0, uint32_t k1) {
        if (k1 - k0 > kLong) {
            met_long = true;
            return;
        }
        df acc[V];
        pull_row_sum<KB, V>(acc, lo + r, k0, k1, part, lrow, lint, x, ldx, lane, pf);
#pragma unroll
        for (int v = 0; v < V; v++) c[(int64_t)r * KB + lane * V + v] = df_val(acc[v]);
    };
#pragma unroll
    for (int j = 0; j < PF; j++) {
        const int r = g + j * NG;
        if (r < cnt) group_row(r, kr[j][0], kr[j][1]);
    }
    for (int r = g + PF * NG; r < cnt; r += NG) {
        uint32_t k0, k1;
        row_range(r, k0, k1);
        group_row(r, k0, k1);
    }
    // the long rows (rare: hubs of a power-law graph), each by the whole CTA:
    // every group sums a strided share, the groups of a warp combine by a
    // fixed shuffle tree, then one thread per right-hand side adds the warps
    // in order (deterministic)
    if (__syncthreads_or(met_long)) {
        constexpr int kMaskWords = (kPullMaxTile + kHalo + 31) / 32;
        __shared__ uint32_t long_mask[kMaskWords];
        const int mwords = (cnt + 31) / 32;
        for (int t = threadIdx.x; t < mwords; t += blockDim.x) long_mask[t] = 0u;
        __syncthreads();
        for (int r = threadIdx.x; r < cnt; r += blockDim.x) {
            uint32_t k0, k1;
            row_range(r, k0, k1);
            if (k1 - k0 > kLong) atomicOr(&long_mask[r >> 5], 1u << (r & 31));
        }
        __syncthreads();
        constexpr int NWmax = 256 / 32;
        __shared__ df long_part[NWmax][KB];
        const int lane32 = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
        for (int wd = 0; wd < mwords; wd++) {
            for (uint32_t bits = long_mask[wd]; bits; bits &= bits - 1) {
                const int r = wd * 32 + __ffs(bits) - 1;
                uint32_t k0, k1;
                row_range(r, k0, k1);
                df acc[V];
#pragma unroll
                for (int v = 0; v < V; v++) acc[v] = df_zero();
                pull_row_entries<KB, V>(acc, k0 + (uint32_t)g, k1, (uint32_t)NG, part, lane);
#pragma unroll
                for (int v = 0; v < V; v++)
                    for (int o = G; o < 32; o <<= 1) acc[v] = df_add(acc[v], df_shfl_xor(acc[v], o));
                if (lane32 < G) {
#pragma unroll
                    for (int v = 0; v < V; v++) long_part[warp][lane32 * V + v] = acc[v];
                }
                __syncthreads();
                if (threadIdx.x < KB) {
                    df t[1] = {df_zero()};
                    for (int w = 0; w < NW; w++) t[0] = df_add(t[0], long_part[w][threadIdx.x]);
                    pull_row_intervals<KB, 1>(t, lo + r, lrow, lint, x, ldx, threadIdx.x, pf);
                    c[(int64_t)r * KB + threadIdx.x] = df_val(t[0]);
                }
                __syncthreads();
            }
        }
    }

    auto emit = [&](int r, const int (&ix)[kMaxChain + 1], int len) {
        Vec<V> out;
#pragma unroll
        for (int v = 0; v < V; v++) {
            df sacc = {c[(int64_t)ix[len - 1] * KB + lane * V + v], 0.f};
            for (int t = len - 2; t >= 0; t--) sacc = df_addf(sacc, c[(int64_t)ix[t] * KB + lane * V + v]);
            out.v[v] = df_val(sacc);
        }
        stv<V>(y + (lo + r) * ldy + lane * V, out);
    };
#pragma unroll
    for (int j = 0; j < PF; j++)
        if (clen[j] > 0) emit(own0 + g + j * NG, idx[j], clen[j]);
    for (int r = own0 + g + PF * NG; r < cnt; r += NG) {
        int ix[kMaxChain + 1];
        const int len = pull_chain_of(meta, lo, r, ix);
        emit(r, ix, len);
    }
}

// ---------------------------------------------------------------------------
// Push, chain step: z_k = sum of x_i over the rows i whose reference chain
// passes through k (Proposition 1 read for the left product: v_i is the sum
// of the difference rows along its chain), i.e. x summed over the subtree of
// k in the reference forest. desc[k] bit t marks row k + t + 1 as a
// descendant (a chain spans at most kHalo rows). A CTA owns ChainShape::TILE
// rows; it stages x for its rows and kHalo rows past the end in shared
// memory, reads the masks of its own rows into registers (all loads of a
// thread are independent and issued together), then each row adds its
// descendants in increasing row order into a compensated (hi, lo) sum:
// bit-reproducible, one barrier. Optionally x is scaled per row first
// (x_i * rowscale_i, PageRank's 1/outdeg). The kernel allows the next
// kernel on the stream to launch early (programmatic dependent launch).
// ---------------------------------------------------------------------------
template <int KB, int V>
struct ChainShape {
    static constexpr int NT = 256;
    static constexpr int G = KB / V;
    static constexpr int NG = NT / G;
    static constexpr int TILE = 4096 / KB > 1024 ? 1024 : (4096 / KB < 128 ? 128 : 4096 / KB);
    static constexpr int RPT = TILE / NG;  // rows per group
};

// One tile of the chain step (rows [blk * TILE, blk * TILE + TILE) of a graph
// with n rows); shared by the one-graph and the multi-graph kernels.
template <int KB, int V>
__device__ __forceinline__ void chain_tile(int64_t blk, const uint32_t* __restrict__ desc,
                                           const float* __restrict__ x, int64_t ldx,
                                           const float* __restrict__ rowscale, float* __restrict__ z, int64_t ldz,
                                           int64_t n) {
    using Sh = ChainShape<KB, V>;
    constexpr int G = Sh::G, NG = Sh::NG, TILE = Sh::TILE, RPT = Sh::RPT;
    __shared__ float xs[(TILE + kHalo) * KB];
    const int g = threadIdx.x / G, lane = threadIdx.x % G;
    const int64_t a = blk * TILE;
    const int cnt = (int)((a + TILE + kHalo < n ? a + TILE + kHalo : n) - a);
    const int own = (int)((a + TILE < n ? a + TILE : n) - a);

    uint32_t m[RPT];
#pragma unroll
    for (int i = 0; i < RPT; i++) {
        const int r = g + i * NG;
        m[i] = r < own ? __ldg(desc + a + r) : 0u;
    }
    for (int r = g; r < cnt; r += NG) {
        Vec<V> xv = ldv<V>(x + (a + r) * ldx + lane * V);
        const float sc = rowscale ? __ldg(rowscale + a + r) : 1.0f;
#pragma unroll
        for (int v = 0; v < V; v++) xs[r * KB + lane * V + v] = __fmul_rn(xv.v[v], sc);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RPT; i++) {
        const int r = g + i * NG;
        if (r >= own) break;
        // the first two descendants as straight-line predicated adds (most
        // rows have at most two), the rest in a short loop
        const uint32_t m1 = m[i], m2 = m1 & (m1 - 1), m3 = m2 & (m2 - 1);
        const int c1 = r + __ffs(m1), c2 = r + __ffs(m2);
        df acc[V];
#pragma unroll
        for (int v = 0; v < V; v++) {
            acc[v] = {xs[r * KB + lane * V + v], 0.f};
            acc[v] = df_addf(acc[v], m1 ? xs[c1 * KB + lane * V + v] : 0.f);
            acc[v] = df_addf(acc[v], m2 ? xs[c2 * KB + lane * V + v] : 0.f);
        }
        for (uint32_t mm = m3; mm; mm &= mm - 1) {
            const int c = r + __ffs(mm);  // bit t -> row r + t + 1
#pragma unroll
            for (int v = 0; v < V; v++) acc[v] = df_addf(acc[v], xs[c * KB + lane * V + v]);
        }
        Vec<V> out;
#pragma unroll
        for (int v = 0; v < V; v++) out.v[v] = df_val(acc[v]);
        stv<V>(z + (a + r) * ldz + lane * V, out);
    }
}

template <int KB, int V>
__global__ void __launch_bounds__(256) k_chain(const uint32_t* __restrict__ desc, const float* __restrict__ x,
                                               int64_t ldx, const float* __restrict__ rowscale,
                                               float* __restrict__ z, int64_t ldz, int64_t n,
                                               const PrState* __restrict__ st) {
    asm volatile("griddepcontrol.launch_dependents;");
    if (st && (__ldcg(&st->done) || __ldcg(&st->iter) >= __ldcg(&st->max_iter))) return;  // PageRank finished
    chain_tile<KB, V>(blockIdx.x, desc, x, ldx, rowscale, z, ldz, n);
}

// ---------------------------------------------------------------------------
// Push, scatter step, written as a gather per column (owner computes, no
// atomics, deterministic): y_j = sum_k z_k A'_kj. The column-major entries of
// column j are +z_k (residual id j of row k), -z_k (dropped id j of row k),
// and interval events: D_j += z_k where an interval of row k starts at j,
// D_j -= z_k where it ends just before j. Intervals contribute the running
// prefix I_j of D. A CTA owns T columns from a, a multiple of kCarryTile, and
// starts I from the intervals open at a (the carry list), so no grid-wide
// scan is needed. A group of G = KB/V lanes owns CPT consecutive columns.
// Each column's first S entries are loaded and summed by the same
// straight-line predicated code in every lane (no divergence on the typical
// column; the entries past them form tail items of at most kTailItem
// entries, handed to the CTA's lane groups evenly, one per group per round,
// so no lane walks a long column while the rest of its warp waits. The point
// terms of a column's first S entries sum in FP32 in storage order (an error
// there stays in y_j, and S is small); the tail items' points (long columns:
// the hubs of a power-law graph) sum compensated. Interval events and their prefix are carried as compensated
// double-float values (two_sum steps, about 48 significant bits), because the
// prefix carries any error to every later column of the tile. The block scan
// runs in the same arithmetic, in a fixed order. y_j = P_j + I_j is rounded
// once.
// The kernel is launched so that it may start while the chain kernel is
// still running (programmatic dependent launch): it reads only the structure
// before griddepcontrol.wait, and reads z afterwards with coherent loads
// (ld.global.ca), never through the read-only non-coherent path, since z
// changes during the kernel's lifetime.
// EPI = 0: store y. EPI = 1: PageRank epilogue (see PrArgs).
// EV = false: the same gather over point columns, where every interval member
// is its own +z_k entry: no events, no carry list, no block scan; y_j is the
// sum of column j's entries alone: the first kPointSlots in FP32, then runs
// of at most kTailItem, each summed in FP32 and joined through an error-free
// two_sum (the error stays near 3u of the column's magnitudes at any
// length). It reads more structure (an interval of length L costs L entries,
// not two) and executes far fewer instructions per right-hand side, which
// wins once a column block carries several right-hand sides.
// ---------------------------------------------------------------------------
template <int KB, int V>
struct GatherShape {
    static constexpr int G = KB / V;                     // lanes per column group
    static constexpr int NT = G >= 8 ? 512 : 256;        // threads per CTA (wide blocks: more, smaller groups)
    static constexpr int NG = NT / G;                    // column groups per CTA
    static constexpr int CPT = 128 / NG > 2 ? 128 / NG : 2;  // consecutive columns per group
    static constexpr int T = NG * CPT;                   // columns per CTA (a multiple of kCarryTile)
    static constexpr int S = kGatherSlots;               // entry slots per column in straight-line code
};

template <int KB>
struct PrPartials {
    double S[KB], R[KB], Dg[KB];
};

// Sums the per-CTA partials (sum q, sum |q - p_prev|, dangling mass): each
// thread's compensated FP32 sums are combined across the CTA in compensated
// FP32 (error-free two_sum steps, fixed order) and stored as one FP64 value
// per CTA. Then two levels, each deterministic and free of spin-waits: the
// last CTA to finish in each group of kPrGroup CTAs adds the group's values in
// FP64 in a fixed order (one warp per quantity, lanes over the CTAs, a fixed
// shuffle tree), and the last group to finish adds the groups' values the same
// way and writes the scalars of this update. A single reducing CTA for the
// whole grid would read grid x 3k values alone (5 MB for k = 32 at n = 862k).
constexpr int kPrGroup = 64;

template <int KB>
__device__ __forceinline__ double pr_warp_sum(const double* __restrict__ base, int count, int item, int lane32) {
    double t = 0.0;
    for (int b = lane32; b < count; b += 32) t += __ldcg(base + ((int64_t)b * 3 + item / KB) * KB + item % KB);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t;
}

// F32WARP: the threads' values are plain FP32 partials (lo = 0) and the
// warp's shuffle tree adds them in FP32 (a few roundings relative to the
// warp's sum of nonnegative terms); the warps are then combined compensated.
template <int KB, int V, bool F32WARP = false>
__device__ df pr_block_sum(df (&S)[V], df (&R)[V], df (&Dg)[V]) {
    // the CTA's sums: thread f * KB + c (< 3 KB) returns quantity f (0: sum
    // q, 1: sum |q - p_prev|, 2: dangling mass) of right-hand side c, every
    // other thread zero; ends on a barrier (the shared array may be reused)
    constexpr int G = KB / V;
    __shared__ df sh_part[32][3][KB];
    const int lane32 = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
#pragma unroll
    for (int v = 0; v < V; v++) {
        for (int o = 16; o >= G; o >>= 1) {
            if constexpr (F32WARP) {
                S[v].hi = __fadd_rn(S[v].hi, __shfl_xor_sync(0xffffffffu, S[v].hi, o));
                R[v].hi = __fadd_rn(R[v].hi, __shfl_xor_sync(0xffffffffu, R[v].hi, o));
                Dg[v].hi = __fadd_rn(Dg[v].hi, __shfl_xor_sync(0xffffffffu, Dg[v].hi, o));
            } else {
                S[v] = df_add(S[v], df_shfl_xor(S[v], o));
                R[v] = df_add(R[v], df_shfl_xor(R[v], o));
                Dg[v] = df_add(Dg[v], df_shfl_xor(Dg[v], o));
            }
        }
    }
    if (lane32 < G) {
#pragma unroll
        for (int v = 0; v < V; v++) {
            sh_part[warp][0][lane32 * V + v] = S[v];
            sh_part[warp][1][lane32 * V + v] = R[v];
            sh_part[warp][2][lane32 * V + v] = Dg[v];
        }
    }
    __syncthreads();
    df t = df_zero();
    if (threadIdx.x < 3 * KB) {
        const int f = threadIdx.x / KB, c = threadIdx.x % KB;
        for (int w = 0; w < NW; w++) t = df_add(t, sh_part[w][f][c]);
    }
    __syncthreads();
    return t;
}

// The grid's sums from each CTA's (pr_block_sum's t, possibly accumulated
// over several tiles), and the update's scalars and state.
template <int KB>
__device__ void pr_grid_sum(df t, const PrArgs& pa, bool init) {
    __shared__ bool sh_last;
    const int lane32 = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
    if (threadIdx.x < 3 * KB) {
        const int f = threadIdx.x / KB, c = threadIdx.x % KB;
        pa.partial[((int64_t)blockIdx.x * 3 + f) * KB + c] = (double)t.hi + (double)t.lo;
        __threadfence();
    }
    __syncthreads();
    // level 1: the last CTA of this group adds the group's CTAs
    const int grp = blockIdx.x / kPrGroup;
    const int gsize = min(kPrGroup, (int)gridDim.x - grp * kPrGroup);
    if (threadIdx.x == 0) sh_last = atomicAdd(pa.gcounter + grp, 1u) == (unsigned)gsize - 1u;
    __syncthreads();
    if (!sh_last) return;
    __threadfence();
    const double* gbase = pa.partial + (int64_t)grp * kPrGroup * 3 * KB;
    for (int item = warp; item < 3 * KB; item += NW) {
        const double t = pr_warp_sum<KB>(gbase, gsize, item, lane32);
        if (lane32 == 0) pa.gpartial[((int64_t)grp * 3 + item / KB) * KB + item % KB] = t;
    }
    __threadfence();
    __syncthreads();
    // level 2: the last group adds the groups and writes the scalars
    const int ngroups = ((int)gridDim.x + kPrGroup - 1) / kPrGroup;
    if (threadIdx.x == 0) {
        pa.gcounter[grp] = 0u;  // every CTA of the group has counted
        sh_last = atomicAdd(pa.counter, 1u) == (unsigned)ngroups - 1u;
    }
    __syncthreads();
    if (!sh_last) return;
    __threadfence();
    __shared__ double sh_tot[3][KB];
    for (int item = warp; item < 3 * KB; item += NW) {
        const double t = pr_warp_sum<KB>(pa.gpartial, ngroups, item, lane32);
        if (lane32 == 0) sh_tot[item / KB][item % KB] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bool conv = true, bad = false;
        for (int c = 0; c < pa.k; c++) {
            const double Ssum = sh_tot[0][c], Rsum = sh_tot[1][c], Dsum = sh_tot[2][c];
            pa.sc_new[0 * KB + c] = 1.0 / Ssum;
            pa.sc_new[1 * KB + c] = Dsum;
            reinterpret_cast<float*>(pa.sc_new + kScDoubles)[c] = (float)Dsum;
            pa.sc_new[2 * KB + c] = init ? INFINITY : Rsum;
            if (!(Rsum < pa.st->tol)) conv = false;
            if (!isfinite(Ssum) || !isfinite(Dsum) || (!init && !isfinite(Rsum)) || Ssum <= 0.0) bad = true;
        }
        if (init) {
            pa.st->iter = 0;
            pa.st->done = bad ? 1 : 0;
            pa.st->numeric = bad ? 1 : 0;
        } else {
            pa.st->iter += 1;
            if (bad) pa.st->numeric = 1;
            if (conv || bad) pa.st->done = 1;
        }
        *pa.counter = 0u;
        if (pa.tile_counter) *pa.tile_counter = 0u;  // every CTA has taken its last tile
        __threadfence();
    }
}

template <int KB, int V, bool F32WARP = false>
__device__ void pr_block_reduce(df (&S)[V], df (&R)[V], df (&Dg)[V], const PrArgs& pa, bool init) {
    pr_grid_sum<KB>(pr_block_sum<KB, V, F32WARP>(S, R, Dg), pa, init);
}

// The FP32 sum sr of one run of point entries [e0, min(e0 + kTailItem, e1))
// (signs applied by an exact FMA with +-1).
template <int V>
__device__ __forceinline__ void point_run(float (&sr)[V], uint32_t e0, uint32_t e1, const uint32_t* __restrict__ ent,
                                          const float* z, int64_t ldz, int lane) {
    const uint32_t cnt = e1 - e0;
    uint32_t we[kTailItem];
#pragma unroll
    for (int t = 0; t < kTailItem; t++) we[t] = (uint32_t)t < cnt ? __ldg(ent + e0 + t) : 0u;
    Vec<V> zc[kTailItem];
#pragma unroll
    for (int t = 0; t < kTailItem; t++) {
#pragma unroll
        for (int v = 0; v < V; v++) zc[t].v[v] = 0.f;
        if ((uint32_t)t < cnt) zc[t] = ldv_ca<V>(z + (int64_t)id_of(we[t]) * ldz + lane * V);
    }
#pragma unroll
    for (int v = 0; v < V; v++) sr[v] = 0.f;
#pragma unroll
    for (int t = 0; t < kTailItem; t++) {
        const float sg = (we[t] >> kIdBits) & 1 ? -1.f : 1.f;  // sg * z is exact
#pragma unroll
        for (int v = 0; v < V; v++) sr[v] = __fmaf_rn(sg, zc[t].v[v], sr[v]);
    }
}

// One tile of the gather (columns [blk * T, blk * T + T)); shared by the
// one-graph and the multi-graph kernels.
// Returns false when a PageRank update finds the iteration finished (past
// convergence or max_iter: nothing done); EPI = 1 adds the tile's block sums
// (pr_block_sum) into acc.
template <int KB, int V, int EPI, bool EV>
__device__ __forceinline__ bool gather_tile(int64_t blk, const uint32_t* __restrict__ colp,
                                            const uint32_t* __restrict__ tent,
                                            const uint32_t* __restrict__ titem_ptr,
                                            const uint32_t* __restrict__ titem,
                                            const uint32_t* __restrict__ carry_ptr,
                                            const uint32_t* __restrict__ carry,
                                            const uint8_t* __restrict__ long_chunk, const float* z, int64_t ldz,
                                            float* __restrict__ y, int64_t ldy, int64_t n, const PrArgs& pa,
                                            df& acc) {
    using Sh = GatherShape<KB, V>;
    constexpr int G = Sh::G, T = Sh::T, CPT = Sh::CPT, NT = Sh::NT, NW = NT / 32;
    constexpr int S = EV ? Sh::S : kPointSlots;
    static_assert(T % kCarryTile == 0, "tile must align with the carry lists");
    static_assert(NW * KB <= NT, "one thread per (warp, right-hand side) forms the warp prefixes");
    __shared__ df run_s[KB];
    __shared__ df wtot_s[NW][KB];
    __shared__ df wpre_s[NW][KB];
    const int g = threadIdx.x / G, lane = threadIdx.x % G;
    const int lane32 = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t a = blk * T;
    const int64_t end = a + T < n ? a + T : n;
    const int64_t c0 = a + (int64_t)g * CPT;

    // structure loads do not depend on the previous kernel: issue them first
    uint32_t cp[CPT + 1], ip[CPT + 1];
#pragma unroll
    for (int q = 0; q <= CPT; q++) {
        cp[q] = __ldg(colp + (c0 + q < end ? c0 + q : end));
        ip[q] = __ldg(titem_ptr + (c0 + q < end ? c0 + q : end));
    }
    const uint32_t it0 = __ldg(titem_ptr + a), it1 = __ldg(titem_ptr + end);  // the tile's tail items
    // point columns, lane groups of several lanes: a column with more than
    // kLongColumn tail entries (a hub of a graph with power-law in-degree) is
    // summed by the whole CTA; the layout flags the 128-column chunks that
    // hold one, so other tiles pay nothing for it
    bool tile_long = false;
    if constexpr (!EV && G > 1) {
#pragma unroll
        for (int c = 0; c < T / kCarryTile; c++)
            if (a + (int64_t)c * kCarryTile < n) tile_long |= __ldg(long_chunk + a / kCarryTile + c) != 0;
    }
    uint32_t cr0 = 0, cr1 = 0, csrc = 0;
    if constexpr (EV) {
        const int64_t ct = a / kCarryTile;
        cr0 = __ldg(carry_ptr + ct);
        cr1 = __ldg(carry_ptr + ct + 1);
        // carry sources of this tile (warp 0; the first 32 now, any further ones later)
        csrc = (warp == 0 && cr0 + lane32 < cr1) ? __ldg(carry + cr0 + lane32) : 0u;
    }
    uint32_t w[CPT][S];
#pragma unroll
    for (int q = 0; q < CPT; q++)
#pragma unroll
        for (int t = 0; t < S; t++) w[q][t] = cp[q] + t < cp[q + 1] ? __ldg(tent + cp[q] + t) : 0u;
    // PageRank epilogue inputs: the previous iterate was written by the
    // previous update, which completed before this update's chain kernel
    // started, and the teleport vectors and 1/outdeg never change; so they
    // are fetched before the wait too (into registers for one right-hand
    // side, into L2 otherwise, where registers are scarce)
    constexpr bool kPfRegs = EPI == 1 && KB == 1;
    float io_pf[CPT], qp_pf[CPT], p0_pf[CPT];
    if constexpr (EPI == 1) {
#pragma unroll
        for (int q = 0; q < CPT; q++) {
            const int64_t j = c0 + q;
            if (j >= end) continue;
            if constexpr (kPfRegs) {
                io_pf[q] = __ldg(pa.inv_outdeg + j);
                qp_pf[q] = __ldg(pa.q_prev + j * pa.ldq);
                p0_pf[q] = pa.p0 ? __ldg(pa.p0 + j * pa.ldp0) : 0.f;
            } else {
                asm volatile("prefetch.global.L2 [%0];" ::"l"(pa.q_prev + j * pa.ldq + lane * V));
                if (pa.p0) asm volatile("prefetch.global.L2 [%0];" ::"l"(pa.p0 + j * pa.ldp0 + lane * V));
            }
        }
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");  // z (and the PageRank state) are ready
    if constexpr (EPI == 1) {
        if (__ldcg(&pa.st->done) || __ldcg(&pa.st->iter) >= __ldcg(&pa.st->max_iter)) return false;
    }

    // running interval sum at column a: the carry sources' z, one thread per
    // right-hand side for a wide column block, the lanes of warp 0 otherwise
    if constexpr (!EV) {
    } else if constexpr (KB >= 8) {
        if (threadIdx.x < KB) {
            df acc = df_zero();
            for (uint32_t e = cr0; e < cr1; e++) {
                const uint32_t src = __ldg(carry + e);
                acc = df_addf(acc, __ldca(z + (int64_t)src * ldz + threadIdx.x));
            }
            run_s[threadIdx.x] = acc;
        }
    } else if (warp == 0) {
        df acc[KB];
#pragma unroll
        for (int c = 0; c < KB; c++) acc[c] = df_zero();
        if (cr0 + lane32 < cr1) {
            const float* zr = z + (int64_t)csrc * ldz;
#pragma unroll
            for (int c = 0; c < KB; c++) acc[c] = df_addf(acc[c], __ldca(zr + c));
        }
        for (uint32_t e = cr0 + 32 + lane32; e < cr1; e += 32) {  // rare: more than 32 open intervals
            const float* zr = z + (int64_t)__ldg(carry + e) * ldz;
#pragma unroll
            for (int c = 0; c < KB; c++) acc[c] = df_addf(acc[c], __ldca(zr + c));
        }
#pragma unroll
        for (int c = 0; c < KB; c++) {
            for (int o = 16; o > 0; o >>= 1) acc[c] = df_add_rn(acc[c], df_shfl_xor(acc[c], o));
            if (lane32 == 0) run_s[c] = acc[c];
        }
    }

    // one pass over each column's entries: the first S points in FP32, points
    // past them (long columns: hubs of a power-law graph reach hundreds) and
    // all events compensated
    float P[CPT][V], Pe[CPT][V];  // Pe: the error terms of the compensated point sum of long columns
    df D[CPT][V], tot[V];
#pragma unroll
    for (int v = 0; v < V; v++) tot[v] = df_zero();
#pragma unroll
    for (int q = 0; q < CPT; q++) {
#pragma unroll
        for (int v = 0; v < V; v++) {
            P[q][v] = 0.f;
            Pe[q][v] = 0.f;
            D[q][v] = df_zero();
        }
#pragma unroll
        for (int t = 0; t < S; t++) {
            const bool valid = cp[q] + t < cp[q + 1];
            Vec<V> zv;
#pragma unroll
            for (int v = 0; v < V; v++) zv.v[v] = 0.f;
            if (valid) zv = ldv_ca<V>(z + (int64_t)id_of(w[q][t]) * ldz + lane * V);
            const uint32_t tag = w[q][t] >> kIdBits;
            if constexpr (EV) {
                const bool point = tag < 2;
#pragma unroll
                for (int v = 0; v < V; v++) {
                    const float val = (tag & 1) ? -zv.v[v] : zv.v[v];
                    P[q][v] += point ? val : 0.f;
                    if (!point) D[q][v] = df_addf(D[q][v], val);
                }
            } else {
                const float sg = (tag & 1) ? -1.f : 1.f;  // sg * z is exact: the same rounding as P -+ z
#pragma unroll
                for (int v = 0; v < V; v++) P[q][v] = __fmaf_rn(sg, zv.v[v], P[q][v]);
            }
        }
    }

    // tail items (entries past a column's first S). With one lane per column
    // group the items are shared out: one item per group per round, its point
    // and event partial sums in shared memory, then each column adds the
    // items of the round that are its own, in order. With several lanes per
    // group (wide column blocks) each group reads its own columns' items in
    // order instead (no extra barriers, fewer registers).
    if constexpr (G > 1 && !EV) {
        // point columns: the entries past the first S in runs of kTailItem,
        // straight from the column (no item table); a run sums in FP32 (its
        // error is at most 3u of its magnitudes) and joins the column's sum
        // through one error-free two_sum, so the column's error stays near 3u
        // of its magnitudes however long it is
#pragma unroll
        for (int q = 0; q < CPT; q++) {
            if (cp[q + 1] > cp[q] + S + kLongColumn) continue;  // left for the whole CTA below
            for (uint32_t e0 = cp[q] + S; e0 < cp[q + 1]; e0 += kTailItem) {
                float sr[V];
                point_run<V>(sr, e0, cp[q + 1], tent, z, ldz, lane);
#pragma unroll
                for (int v = 0; v < V; v++) {
                    float s_, e_;
                    two_sum(P[q][v], sr[v], s_, e_);
                    P[q][v] = s_;
                    Pe[q][v] = __fadd_rn(Pe[q][v], e_);
                }
            }
        }
        // long columns, each by the whole CTA: every group sums a strided
        // share of the entries, the groups of a warp combine by a fixed
        // shuffle tree and one thread per right-hand side adds the warps in
        // order (deterministic); the owning group adds the result to its column
        if (tile_long) {  // the same in every thread of the CTA
            constexpr int NWl = NT / 32;
            __shared__ uint32_t long_mask[(T + 31) / 32];
            __shared__ df long_part[NWl][KB];
            __shared__ df long_res[KB];
            for (int t = threadIdx.x; t < (T + 31) / 32; t += NT) long_mask[t] = 0u;
            __syncthreads();
#pragma unroll
            for (int q = 0; q < CPT; q++)
                if (lane == 0 && cp[q + 1] > cp[q] + S + kLongColumn) {
                    const int cc = g * CPT + q;
                    atomicOr(&long_mask[cc >> 5], 1u << (cc & 31));
                }
            __syncthreads();
            for (int wd = 0; wd < (T + 31) / 32; wd++) {
                for (uint32_t bits = long_mask[wd]; bits; bits &= bits - 1) {
                    const int cc = wd * 32 + __ffs(bits) - 1;
                    const uint32_t eb = __ldg(colp + a + cc) + S, ee = __ldg(colp + a + cc + 1);
                    df acc[V];
#pragma unroll
                    for (int v = 0; v < V; v++) acc[v] = df_zero();
                    // one entry per group and step (few registers: this path
                    // must not raise the register need of the common one)
                    for (uint32_t e = eb + (uint32_t)g; e < ee; e += (uint32_t)(NT / G)) {
                        const uint32_t we = __ldg(tent + e);
                        const Vec<V> zv = ldv_ca<V>(z + (int64_t)id_of(we) * ldz + lane * V);
                        const float sg = (we >> kIdBits) & 1 ? -1.f : 1.f;
#pragma unroll
                        for (int v = 0; v < V; v++) acc[v] = df_addf(acc[v], sg * zv.v[v]);
                    }
#pragma unroll
                    for (int v = 0; v < V; v++)
                        for (int o = G; o < 32; o <<= 1) acc[v] = df_add(acc[v], df_shfl_xor(acc[v], o));
                    if (lane32 < G) {
#pragma unroll
                        for (int v = 0; v < V; v++) long_part[warp][lane32 * V + v] = acc[v];
                    }
                    __syncthreads();
                    if (threadIdx.x < KB) {
                        df t = df_zero();
                        for (int w = 0; w < NWl; w++) t = df_add(t, long_part[w][threadIdx.x]);
                        long_res[threadIdx.x] = t;
                    }
                    __syncthreads();
                    // every thread, predicated (a runtime column index here
                    // would move P and Pe to local memory): two_sum of P with
                    // 0 leaves P and Pe unchanged
#pragma unroll
                    for (int q = 0; q < CPT; q++) {
                        const bool mine = g * CPT + q == cc;
#pragma unroll
                        for (int v = 0; v < V; v++) {
                            const df r = long_res[lane * V + v];
                            float s_, e_;
                            two_sum(P[q][v], mine ? r.hi : 0.f, s_, e_);
                            P[q][v] = s_;
                            Pe[q][v] = __fadd_rn(Pe[q][v], mine ? __fadd_rn(e_, r.lo) : e_);
                        }
                    }
                }
            }
        }
    } else if constexpr (G > 1) {
#pragma unroll
        for (int q = 0; q < CPT; q++) {
            for (uint32_t k = ip[q]; k < ip[q + 1]; k++) {
                const uint32_t wi = __ldg(titem + k);
                const uint32_t e0 = wi & 0x3fffffffu, cnt = (wi >> 30) + 1u;
                uint32_t we[kTailItem];
#pragma unroll
                for (int t = 0; t < kTailItem; t++) we[t] = (uint32_t)t < cnt ? __ldg(tent + e0 + t) : 0u;
                Vec<V> zc[kTailItem];
#pragma unroll
                for (int t = 0; t < kTailItem; t++) {
#pragma unroll
                    for (int v = 0; v < V; v++) zc[t].v[v] = 0.f;
                    if ((uint32_t)t < cnt) zc[t] = ldv_ca<V>(z + (int64_t)id_of(we[t]) * ldz + lane * V);
                }
#pragma unroll
                for (int t = 0; t < kTailItem; t++) {
                    if ((uint32_t)t >= cnt) break;
                    const uint32_t tag = we[t] >> kIdBits;
#pragma unroll
                    for (int v = 0; v < V; v++) {
                        const float val = (tag & 1) ? -zc[t].v[v] : zc[t].v[v];
                        if (!EV || tag < 2) {
                            float s_, e_;
                            two_sum(P[q][v], val, s_, e_);  // the point sum continues compensated
                            P[q][v] = s_;
                            Pe[q][v] = __fadd_rn(Pe[q][v], e_);
                        } else {
                            D[q][v] = df_addf(D[q][v], val);
                        }
                    }
                }
            }
        }
    } else {
        constexpr int NGR = NT / G;  // items per round
        __shared__ df tail_pt[NGR][KB], tail_ev[NGR][EV ? KB : 1];
        for (uint32_t r0 = it0; r0 < it1; r0 += NGR) {  // the same trip count in every thread
            const uint32_t i = r0 + (uint32_t)g;
            if (i < it1) {
                const uint32_t wi = __ldg(titem + i);
                const uint32_t e0 = wi & 0x3fffffffu, cnt = (wi >> 30) + 1u;
                uint32_t we[kTailItem];
#pragma unroll
                for (int t = 0; t < kTailItem; t++) we[t] = (uint32_t)t < cnt ? __ldg(tent + e0 + t) : 0u;
                Vec<V> zc[kTailItem];
#pragma unroll
                for (int t = 0; t < kTailItem; t++) {
#pragma unroll
                    for (int v = 0; v < V; v++) zc[t].v[v] = 0.f;
                    if ((uint32_t)t < cnt) zc[t] = ldv_ca<V>(z + (int64_t)id_of(we[t]) * ldz + lane * V);
                }
                df pt[V], ev[V];
#pragma unroll
                for (int v = 0; v < V; v++) pt[v] = ev[v] = df_zero();
#pragma unroll
                for (int t = 0; t < kTailItem; t++) {
                    const uint32_t tag = we[t] >> kIdBits;
                    const bool point = !EV || tag < 2;
#pragma unroll
                    for (int v = 0; v < V; v++) {
                        const float val = (tag & 1) ? -zc[t].v[v] : zc[t].v[v];
                        if constexpr (EV) {
                            pt[v] = df_addf(pt[v], point ? val : 0.f);
                            ev[v] = df_addf(ev[v], point ? 0.f : val);
                        } else {
                            pt[v].hi = __fadd_rn(pt[v].hi, val);  // a run of at most kTailItem sums in FP32
                        }
                    }
                }
#pragma unroll
                for (int v = 0; v < V; v++) {
                    tail_pt[g][lane * V + v] = pt[v];
                    if constexpr (EV) tail_ev[g][lane * V + v] = ev[v];
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < CPT; q++) {
                const uint32_t b = ip[q] > r0 ? ip[q] : r0;
                const uint32_t e = ip[q + 1] < r0 + NGR ? ip[q + 1] : r0 + NGR;
                for (uint32_t k = b; k < e; k++) {
#pragma unroll
                    for (int v = 0; v < V; v++) {
                        const df tp = tail_pt[k - r0][lane * V + v];
                        float s_, e_;
                        two_sum(P[q][v], tp.hi, s_, e_);  // the point sum continues compensated
                        P[q][v] = s_;
                        Pe[q][v] = __fadd_rn(Pe[q][v], __fadd_rn(e_, tp.lo));
                        if constexpr (EV) D[q][v] = df_add_rn(D[q][v], tail_ev[k - r0][lane * V + v]);
                    }
                }
            }
            // the next round overwrites the item sums; after the last round
            // nothing does (the same condition in every thread)
            if (r0 + NGR < it1) __syncthreads();
        }
    }
    // exclusive prefix of the group totals across the block (event columns only)
    df run[V];
#pragma unroll
    for (int v = 0; v < V; v++) run[v] = df_zero();
    if constexpr (EV) {
#pragma unroll
    for (int q = 0; q < CPT; q++)
#pragma unroll
        for (int v = 0; v < V; v++) tot[v] = df_add_rn(tot[v], D[q][v]);

    // exclusive prefix of the group totals across the block, in a fixed order:
    // carry, then the warps before this one, then the groups before this one
    df inc[V];
#pragma unroll
    for (int v = 0; v < V; v++) inc[v] = tot[v];
#pragma unroll
    for (int d = G; d < 32; d <<= 1)
#pragma unroll
        for (int v = 0; v < V; v++) {
            const df o = df_shfl_up(inc[v], d);
            if (lane32 >= d) inc[v] = df_add_rn(o, inc[v]);
        }
    if (lane32 >= 32 - G) {
#pragma unroll
        for (int v = 0; v < V; v++) wtot_s[warp][lane * V + v] = inc[v];
    }
    df excl[V];
#pragma unroll
    for (int v = 0; v < V; v++) {
        const df o = df_shfl_up(inc[v], G);
        excl[v] = lane32 >= G ? o : df_zero();
    }
    __syncthreads();
    // this warp's starting prefix: the carry, then the totals of the warps
    // before it, in order; for a wide column block formed once per (warp,
    // right-hand side) in shared memory, otherwise by every thread (cheaper
    // than a second barrier when each thread owns few right-hand sides)
    if constexpr (KB >= 8) {
        if (threadIdx.x < NW * KB) {
            const int w = threadIdx.x / KB, c = threadIdx.x % KB;
            df r = run_s[c];
            for (int w2 = 0; w2 < w; w2++) r = df_add_rn(r, wtot_s[w2][c]);
            wpre_s[w][c] = r;
        }
        __syncthreads();
#pragma unroll
        for (int v = 0; v < V; v++) run[v] = df_add_rn(wpre_s[warp][lane * V + v], excl[v]);
    } else {
        // the earlier warps' totals by a fixed shuffle tree: group gi of this
        // warp holds warp gi's total (when gi < warp), three levels add the
        // eight groups, and group 0's sum is taken by every group
        static_assert(NW == 8 && 32 / G >= NW, "eight warps, at least eight lane groups per warp");
        const int gi = lane32 / G;
#pragma unroll
        for (int v = 0; v < V; v++) {
            df t = gi < warp ? wtot_s[gi][lane * V + v] : df_zero();
#pragma unroll
            for (int o = G; o < NW * G; o <<= 1) t = df_add_rn(t, df_shfl_xor(t, o));
            t.hi = __shfl_sync(0xffffffffu, t.hi, lane);
            t.lo = __shfl_sync(0xffffffffu, t.lo, lane);
            run[v] = df_add_rn(df_add_rn(run_s[lane * V + v], t), excl[v]);
        }
    }
    }  // EV

    // PageRank sums of this thread's CPT columns and then of its warp: plain
    // FP32 adds (a few roundings, relative to partial sums of nonnegative
    // terms), then compensated across the warps of the block
    float Ssum[V], R[V], Dg[V];
    float dl[V];     // the previous update's dangling mass, per right-hand side of this lane
    int64_t sd[V];   // one-hot teleport nodes of this lane's right-hand sides
    const float un = EPI == 1 ? 1.0f / (float)n : 0.0f;  // (an int64 conversion: once, not per column)
#pragma unroll
    for (int v = 0; v < V; v++) {
        Ssum[v] = R[v] = Dg[v] = 0.f;
        if constexpr (EPI == 1) {
            dl[v] = sc_dangling_f32(pa.sc_prev, lane * V + v);
            sd[v] = pa.seed ? __ldg(pa.seed + lane * V + v) : -1;
        }
    }
#pragma unroll
    for (int q = 0; q < CPT; q++) {
        const int64_t j = c0 + q;
        Vec<V> out;
#pragma unroll
        for (int v = 0; v < V; v++) {
            if constexpr (EV) {
                run[v] = df_add_rn(run[v], D[q][v]);
                out.v[v] = df_val(df_addf(df_addf(run[v], P[q][v]), Pe[q][v]));
            } else {
                out.v[v] = __fadd_rn(P[q][v], Pe[q][v]);
            }
        }
        if (j >= end) continue;
        if constexpr (EPI == 0) {
            stv<V>(y + j * ldy + lane * V, out);
        } else {
            float io;
            Vec<V> qp, qn, p0v;
            if constexpr (kPfRegs) {
                io = io_pf[q];
                qp.v[0] = qp_pf[q];
                p0v.v[0] = p0_pf[q];
            } else {
                io = __ldg(pa.inv_outdeg + j);
                qp = ldv<V>(pa.q_prev + j * pa.ldq + lane * V);
                if (pa.p0) p0v = ldv<V>(pa.p0 + j * pa.ldp0 + lane * V);
            }
#pragma unroll
            for (int v = 0; v < V; v++) {
                const float p0j = pa.p0 ? p0v.v[v] : pa.seed ? (j == sd[v] ? 1.0f : 0.0f) : un;
                const float gj = pa.dangling_uniform ? un : p0j;
                const float qj = pa.alpha * p0j + (1.0f - pa.alpha) * (out.v[v] + dl[v] * gj);
                qn.v[v] = qj;
                Ssum[v] = __fadd_rn(Ssum[v], qj);
                R[v] = __fadd_rn(R[v], fabsf(__fsub_rn(qj, qp.v[v])));
                if (io == 0.0f) Dg[v] = __fadd_rn(Dg[v], qj);
            }
            stv<V>(pa.q_new + j * pa.ldq + lane * V, qn);
        }
    }
    if constexpr (EPI == 1) {
        df Sd[V], Rd[V], Dd[V];
#pragma unroll
        for (int v = 0; v < V; v++) {
            Sd[v] = {Ssum[v], 0.f};
            Rd[v] = {R[v], 0.f};
            Dd[v] = {Dg[v], 0.f};
        }
        acc = df_add(acc, pr_block_sum<KB, V, true>(Sd, Rd, Dd));
    }
    return true;
}

// A PageRank update's gather: a resident grid, each CTA taking tiles from a
// counter and adding their block sums, then one grid-wide reduction (one per
// CTA instead of one per 128-column tile). The product (EPI = 0): one tile
// per CTA.
template <int KB, int V, int EPI, bool EV>
__device__ __forceinline__ void gather_grid(const uint32_t* __restrict__ colp, const uint32_t* __restrict__ tent,
                                           const uint32_t* __restrict__ titem_ptr,
                                           const uint32_t* __restrict__ titem,
                                           const uint32_t* __restrict__ carry_ptr,
                                           const uint32_t* __restrict__ carry,
                                           const uint8_t* __restrict__ long_chunk, const float* z, int64_t ldz,
                                           float* __restrict__ y, int64_t ldy, int64_t n, const PrArgs& pa) {
    df acc = df_zero();
    if constexpr (EPI == 0) {
        gather_tile<KB, V, EPI, EV>(blockIdx.x, colp, tent, titem_ptr, titem, carry_ptr, carry, long_chunk, z, ldz, y,
                                    ldy, n, pa, acc);
    } else {
        // tiles handed out one at a time (CTAs whose tiles ran long take
        // fewer); each tile's block sums are the same whatever CTA takes it,
        // but which tiles a CTA adds up varies from run to run, so the FP64
        // totals can differ in their last bits
        constexpr int T = GatherShape<KB, V>::T;
        const int64_t tiles = (n + T - 1) / T;
        __shared__ unsigned int sh_tile;
        bool took = false;
        for (;;) {
            if (threadIdx.x == 0) sh_tile = atomicAdd(pa.tile_counter, 1u);
            __syncthreads();
            const int64_t blk = sh_tile;
            __syncthreads();
            if (blk >= tiles) break;
            took = true;
            if (!gather_tile<KB, V, EPI, EV>(blk, colp, tent, titem_ptr, titem, carry_ptr, carry, long_chunk, z, ldz,
                                             y, ldy, n, pa, acc))
                return;  // the same answer in every CTA: no CTA reduces
        }
        if (!took) {
            // no tile left for this CTA: the other CTAs took them all, or the
            // update is past convergence or max_iter (such updates return
            // without resetting the counter, which then holds their fetches);
            // the state tells
            asm volatile("griddepcontrol.wait;" ::: "memory");
            if (__ldcg(&pa.st->done) || __ldcg(&pa.st->iter) >= __ldcg(&pa.st->max_iter)) return;
        }
        pr_grid_sum<KB>(acc, pa, false);
    }
}

template <int KB, int V, int EPI>
__global__ void __launch_bounds__(GatherShape<KB, V>::NT) k_gather(const uint32_t* __restrict__ colp, const uint32_t* __restrict__ tent,
                                                const uint32_t* __restrict__ titem_ptr,
                                                const uint32_t* __restrict__ titem,
                                                const uint32_t* __restrict__ carry_ptr,
                                                const uint32_t* __restrict__ carry, const float* z, int64_t ldz,
                                                float* __restrict__ y, int64_t ldy, int64_t n,
                                                PrArgs pa) {
    gather_grid<KB, V, EPI, true>(colp, tent, titem_ptr, titem, carry_ptr, carry, nullptr, z, ldz, y, ldy, n, pa);
}

// The gather over point columns (gather_tile with EV = false)
// (registers capped for 3 resident 512-thread CTAs per SM for the product,
// 2 for the PageRank update, and 4 for 256-thread CTAs: the few spilled bytes
// cost less than the lost occupancy)
template <int KB, int V, int EPI>
__global__ void __launch_bounds__(GatherShape<KB, V>::NT, GatherShape<KB, V>::NT == 512 ? (EPI == 0 ? 3 : 2) : 4)
    k_gather_pt(const uint32_t* __restrict__ colp,
                                                                       const uint32_t* __restrict__ ent,
                                                                       const uint32_t* __restrict__ titem_ptr,
                                                                       const uint32_t* __restrict__ titem,
                                                                       const uint8_t* __restrict__ long_chunk,
                                                                       const float* z, int64_t ldz,
                                                                       float* __restrict__ y, int64_t ldy, int64_t n,
                                                                       PrArgs pa) {
    gather_grid<KB, V, EPI, false>(colp, ent, titem_ptr, titem, nullptr, nullptr, long_chunk, z, ldz, y, ldy, n, pa);
}

// PageRank start: q_0 = p_init (or p0, or the one-hot seeds, or uniform), and the scalars of the
// start (1/S_0, dangling mass) by the same deterministic reduction.
template <int KB, int V>
__global__ void __launch_bounds__(256) k_pr_init(const float* __restrict__ p_init, int64_t ldi, int64_t n,
                                                 int tile, PrArgs pa) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && pa.tile_counter) *pa.tile_counter = 0u;  // a fresh solve
    constexpr int G = KB / V;
    const int NG = blockDim.x / G;
    const int g = threadIdx.x / G, lane = threadIdx.x % G;
    const int64_t a = (int64_t)blockIdx.x * tile;
    const int64_t end = a + tile < n ? a + tile : n;
    df S[V], R[V], Dg[V];
#pragma unroll
    for (int v = 0; v < V; v++) S[v] = R[v] = Dg[v] = df_zero();
    const float un = 1.0f / (float)n;
    for (int64_t j = a + g; j < end; j += NG) {
        Vec<V> pv;
        if (p_init) pv = ldv<V>(p_init + j * ldi + lane * V);
        else if (pa.seed) {
#pragma unroll
            for (int v = 0; v < V; v++) pv.v[v] = j == __ldg(pa.seed + lane * V + v) ? 1.0f : 0.0f;
        } else {
#pragma unroll
            for (int v = 0; v < V; v++) pv.v[v] = un;
        }
        stv<V>(pa.q_new + j * pa.ldq + lane * V, pv);
        const float io = __ldg(pa.inv_outdeg + j);
        if (pa.x_new) {
            Vec<V> xv;
#pragma unroll
            for (int v = 0; v < V; v++) xv.v[v] = __fmul_rn(pv.v[v], io);
            stv<V>(pa.x_new + j * pa.ldq + lane * V, xv);
        }
#pragma unroll
        for (int v = 0; v < V; v++) {
            S[v] = df_addf(S[v], pv.v[v]);
            if (io == 0.0f) Dg[v] = df_addf(Dg[v], pv.v[v]);
        }
    }
    pr_block_reduce<KB, V>(S, R, Dg, pa, true);
}

// p_out = q_T / S_T for the final update T (read from the state): 1/S_T
// rounded to FP32 once per right-hand side, each value scaled in FP32 (FP64
// arithmetic runs at a small fraction of the FP32 rate on this part).
template <int KB, int V>
__global__ void k_pr_final(const float* __restrict__ q0, const float* __restrict__ q1, int64_t ldq,
                           const double* __restrict__ sc0, const double* __restrict__ sc1,
                           const PrState* __restrict__ st, float* __restrict__ out, int64_t ldo, int64_t n) {
    constexpr int G = KB / V;
    const int par = __ldcg(&st->iter) & 1;
    const float* q = par ? q1 : q0;
    const double* sc = par ? sc1 : sc0;
    const int64_t gid = (int64_t)blockIdx.x * (blockDim.x / G) + threadIdx.x / G;
    const int lane = threadIdx.x % G;
    const int64_t stride = (int64_t)gridDim.x * (blockDim.x / G);
    float scv[V];
#pragma unroll
    for (int v = 0; v < V; v++) scv[v] = (float)__ldcg(sc + lane * V + v);
    for (int64_t j = gid; j < n; j += stride) {
        Vec<V> qv = ldv_cg<V>(q + j * ldq + lane * V), o;
#pragma unroll
        for (int v = 0; v < V; v++) o.v[v] = __fmul_rn(qv.v[v], scv[v]);
        stv<V>(out + j * ldo + lane * V, o);
    }
}

}  // namespace bvg

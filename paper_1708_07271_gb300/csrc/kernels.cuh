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

struct PrArgs {
    const float* p0;           // teleport vectors (n x k, ld ldp0) or NULL = uniform 1/n
    int64_t ldp0;
    const float* inv_outdeg;   // 0 marks a row without successors
    const float* q_prev;       // previous iterate, unnormalised (n x k, ld ldq)
    float* q_new;
    float* x_new;              // q_new / outdeg (the next update's input), or NULL
    int64_t ldq;
    const double* sc_prev;     // [3][k]: 1/S, dangling mass, resid (of the previous update)
    double* sc_new;
    PrState* st;
    double* partial;           // [grid][3][KB]
    unsigned int* counter;
    float alpha;
    int dangling_uniform;
    int k;                     // right-hand sides of the solve (== KB)
};


// ---------------------------------------------------------------------------
// Pull: y = A x^T (Sec. 4). A CTA owns rows [a, a + tile). It first forms the
// correction sums c_i = sum_j A'_ij x_j for rows [a - kHalo, a + tile) into
// shared memory (dropped ids subtract, residual ids add, an interval (s, len)
// adds x_s + ... + x_{s+len-1}), then resolves each owned row's chain
// y_i = c_i + y_{r_i} = c_i + c_{r_i} + c_{r_{r_i}} + ... with at most
// max_chain links, all inside the CTA (a chain never leaves kHalo rows).
// The sums are compensated (hi, lo) pairs; the chain is added from its root
// outwards, i.e. in the association of the sequential algorithm.
// ---------------------------------------------------------------------------
template <int KB, int V>
__global__ void __launch_bounds__(256) k_pull(const uint8_t* __restrict__ meta, const uint32_t* __restrict__ rowp,
                                              const uint32_t* __restrict__ ent, const float* __restrict__ x,
                                              int64_t ldx, float* __restrict__ y, int64_t ldy, int64_t n, int tile) {
    constexpr int G = KB / V;
    extern __shared__ float4 smem_pull[];
    df* c = reinterpret_cast<df*>(smem_pull);  // [(tile + kHalo) * KB]
    const int NG = blockDim.x / G;
    const int g = threadIdx.x / G, lane = threadIdx.x % G;
    const int64_t a = (int64_t)blockIdx.x * tile;
    const int64_t lo = a > kHalo ? a - kHalo : 0;
    const int64_t hi = a + tile < n ? a + tile : n;
    const int cnt = (int)(hi - lo);

    for (int r = g; r < cnt; r += NG) {
        const int64_t i = lo + r;
        df acc[V];
#pragma unroll
        for (int v = 0; v < V; v++) acc[v] = df_zero();
        const uint32_t w0 = __ldg(rowp + i), w1 = __ldg(rowp + i + 1);
        for (uint32_t w = w0; w < w1; w++) {
            const uint32_t word = __ldg(ent + w);
            const uint32_t tag = tag_of(word), id = id_of(word);
            if (tag == kTagPlus || tag == kTagMinus) {
                Vec<V> xv = ldv<V>(x + (int64_t)id * ldx + lane * V);
#pragma unroll
                for (int v = 0; v < V; v++) acc[v] = df_addf(acc[v], tag == kTagPlus ? xv.v[v] : -xv.v[v]);
            } else if (tag == kTagIvS) {
                const uint32_t len = id_of(__ldg(ent + w + 1));
                w++;
                for (uint32_t t = 0; t < len; t++) {
                    Vec<V> xv = ldv<V>(x + (int64_t)(id + t) * ldx + lane * V);
#pragma unroll
                    for (int v = 0; v < V; v++) acc[v] = df_addf(acc[v], xv.v[v]);
                }
            }
        }
#pragma unroll
        for (int v = 0; v < V; v++) c[(int64_t)r * KB + lane * V + v] = acc[v];
    }
    __syncthreads();

    for (int r = (int)(a - lo) + g; r < cnt; r += NG) {
        int idx[kMaxChain + 1];
        int len = 0, cur = r;
        idx[len++] = cur;
        for (int t = 0; t < kMaxChain; t++) {
            const int off = __ldg(meta + lo + cur) & 7;
            if (off == 0 || cur - off < 0) break;
            cur -= off;
            idx[len++] = cur;
        }
        Vec<V> out;
#pragma unroll
        for (int v = 0; v < V; v++) {
            df s = c[(int64_t)idx[len - 1] * KB + lane * V + v];
            for (int t = len - 2; t >= 0; t--) s = df_add(c[(int64_t)idx[t] * KB + lane * V + v], s);
            out.v[v] = df_val(s);
        }
        stv<V>(y + (lo + r) * ldy + lane * V, out);
    }
}

// ---------------------------------------------------------------------------
// Push, chain step: z_k = sum of x_i over the rows i whose reference chain
// passes through k (Proposition 1 read for the left product: v_i is the sum
// of the difference rows along its chain), i.e. x summed over the subtree of
// k in the reference forest. desc[k] bit t marks row k + t + 1 as a
// descendant (a chain spans at most kHalo rows), so a CTA that owns rows
// [a, a + tile) stages x for kHalo rows past its end and each row adds its
// descendants in increasing row order into a compensated (hi, lo) sum:
// bit-reproducible, one barrier. Optionally x is scaled per row first
// (x_i * rowscale_i, PageRank's 1/outdeg).
// ---------------------------------------------------------------------------
template <int KB, int V>
__global__ void __launch_bounds__(256) k_chain(const uint32_t* __restrict__ desc, const float* __restrict__ x,
                                               int64_t ldx, const float* __restrict__ rowscale,
                                               float* __restrict__ z, int64_t ldz, int64_t n, int tile,
                                               const PrState* __restrict__ st) {
    if (st && (__ldcg(&st->done) || __ldcg(&st->iter) >= __ldcg(&st->max_iter))) return;  // PageRank finished
    constexpr int G = KB / V;
    extern __shared__ float4 smem_chain[];
    float* xs = reinterpret_cast<float*>(smem_chain);  // [(tile + kHalo) * KB]
    const int NG = blockDim.x / G;
    const int g = threadIdx.x / G, lane = threadIdx.x % G;
    const int64_t a = (int64_t)blockIdx.x * tile;
    const int64_t hi = a + tile + kHalo < n ? a + tile + kHalo : n;
    const int cnt = (int)(hi - a);
    const int own = (int)((a + tile < n ? a + tile : n) - a);

    for (int r = g; r < cnt; r += NG) {
        Vec<V> xv = ldv<V>(x + (a + r) * ldx + lane * V);
        const float sc = rowscale ? __ldg(rowscale + a + r) : 1.0f;
#pragma unroll
        for (int v = 0; v < V; v++) xs[(int64_t)r * KB + lane * V + v] = __fmul_rn(xv.v[v], sc);
    }
    __syncthreads();
    for (int r = g; r < own; r += NG) {
        df acc[V];
#pragma unroll
        for (int v = 0; v < V; v++) acc[v] = {xs[(int64_t)r * KB + lane * V + v], 0.f};
        for (uint32_t m = __ldg(desc + a + r); m; m &= m - 1) {
            const int c = r + __ffs(m);  // bit t -> row r + t + 1
            if (c >= cnt) break;
#pragma unroll
            for (int v = 0; v < V; v++) acc[v] = df_addf(acc[v], xs[(int64_t)c * KB + lane * V + v]);
        }
        Vec<V> out;
#pragma unroll
        for (int v = 0; v < V; v++) out.v[v] = df_val(acc[v]);
        stv<V>(z + (a + r) * ldz + lane * V, out);
    }
}

// ---------------------------------------------------------------------------
// Push, scatter step, written as a gather per column (owner computes, no
// atomics, deterministic): y_j = sum_k z_k A'_kj. The column-major entries of
// column j are +z_k (residual id j of row k), -z_k (dropped id j of row k),
// and interval events: D_j += z_k where an interval of row k starts at j,
// D_j -= z_k where it ends just before j. Intervals contribute the running
// prefix I_j of D. A CTA owns T columns from a, a multiple of kCarryTile, and
// starts I from the intervals open at a (the carry list), so no grid-wide
// scan is needed. A group of G = KB/V lanes owns CPT consecutive columns: it
// sums each column's point entries P_j in FP32 (a few terms in storage order;
// an error there stays in y_j) and its events D_j in compensated (hi, lo)
// form, since the prefix of D carries any error to every later column; the
// prefix runs compensated within the group's columns on the fly and across
// groups by one block scan.
// EPI = 0: store y. EPI = 1: PageRank epilogue (see PrArgs).
// ---------------------------------------------------------------------------
template <int KB, int V>
struct GatherShape {
    static constexpr int NT = 128;                       // threads per CTA
    static constexpr int G = KB / V;                     // lanes per column group
    static constexpr int T = 1024 / KB > 128 ? 1024 / KB : 128;  // columns per CTA
    static constexpr int CPT = T * G / NT;               // columns per group
};

template <int KB>
struct PrPartials {
    double S[KB], R[KB], Dg[KB];
};

// Sums the per-CTA FP64 partials (sum q, sum |q - p_prev|, dangling mass),
// then the last CTA to finish reduces all CTAs in a fixed order and writes
// the scalars of this update (deterministic; no spin-waits).
template <int KB, int V>
__device__ void pr_block_reduce(double (&S)[V], double (&R)[V], double (&Dg)[V], const PrArgs& pa, bool init) {
    constexpr int G = KB / V;
    __shared__ double sh_part[32][3][KB];
    __shared__ bool sh_last;
    const int lane32 = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
#pragma unroll
    for (int v = 0; v < V; v++) {
        for (int o = 16; o >= G; o >>= 1) {
            S[v] += __shfl_xor_sync(0xffffffffu, S[v], o);
            R[v] += __shfl_xor_sync(0xffffffffu, R[v], o);
            Dg[v] += __shfl_xor_sync(0xffffffffu, Dg[v], o);
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
    if (threadIdx.x < 3 * KB) {
        const int f = threadIdx.x / KB, c = threadIdx.x % KB;
        double t = 0.0;
        for (int w = 0; w < NW; w++) t += sh_part[w][f][c];
        pa.partial[((int64_t)blockIdx.x * 3 + f) * KB + c] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) sh_last = atomicAdd(pa.counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!sh_last) return;
    __threadfence();
    __shared__ double sh_red[256];
    __shared__ double sh_tot[3][KB];
    for (int item = 0; item < 3 * KB; item++) {
        double t = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
            t += __ldcg(pa.partial + ((int64_t)b * 3 + item / KB) * KB + item % KB);
        sh_red[threadIdx.x] = t;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) sh_red[threadIdx.x] += sh_red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) sh_tot[item / KB][item % KB] = sh_red[0];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        bool conv = true, bad = false;
        for (int c = 0; c < pa.k; c++) {
            const double Ssum = sh_tot[0][c], Rsum = sh_tot[1][c], Dsum = sh_tot[2][c];
            pa.sc_new[0 * KB + c] = 1.0 / Ssum;
            pa.sc_new[1 * KB + c] = Dsum;
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
        __threadfence();
    }
}

template <int KB, int V, int EPI>
__global__ void __launch_bounds__(128) k_gather(const uint32_t* __restrict__ colp, const uint32_t* __restrict__ tent,
                                                const uint32_t* __restrict__ carry_ptr,
                                                const uint32_t* __restrict__ carry, const float* __restrict__ z,
                                                int64_t ldz, float* __restrict__ y, int64_t ldy, int64_t n,
                                                PrArgs pa) {
    using Sh = GatherShape<KB, V>;
    constexpr int G = Sh::G, T = Sh::T, CPT = Sh::CPT, NT = Sh::NT, NW = NT / 32;
    static_assert(T % kCarryTile == 0, "tile must align with the carry lists");
    if constexpr (EPI == 1) {
        if (__ldcg(&pa.st->done) || __ldcg(&pa.st->iter) >= __ldcg(&pa.st->max_iter)) return;
    }
    __shared__ df run_s[KB];
    __shared__ df wtot_s[NW][KB];
    const int g = threadIdx.x / G, lane = threadIdx.x % G;
    const int lane32 = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t a = (int64_t)blockIdx.x * T;
    const int64_t end = a + T < n ? a + T : n;
    const int64_t c0 = a + (int64_t)g * CPT;

    // running interval prefix at column a: sources of intervals open there
    if (warp == 0) {
        df acc[KB];
#pragma unroll
        for (int c = 0; c < KB; c++) acc[c] = df_zero();
        const int64_t ct = a / kCarryTile;
        const uint32_t e1 = __ldg(carry_ptr + ct + 1);
        for (uint32_t e = __ldg(carry_ptr + ct) + lane32; e < e1; e += 32) {
            const float* zr = z + (int64_t)__ldg(carry + e) * ldz;
#pragma unroll
            for (int c = 0; c < KB; c++) acc[c] = df_addf(acc[c], __ldg(zr + c));
        }
#pragma unroll
        for (int c = 0; c < KB; c++)
            for (int o = 16; o > 0; o >>= 1)
                acc[c] = df_add(acc[c], {__shfl_down_sync(0xffffffffu, acc[c].hi, o),
                                         __shfl_down_sync(0xffffffffu, acc[c].lo, o)});
        if (lane32 == 0) {
#pragma unroll
            for (int c = 0; c < KB; c++) run_s[c] = acc[c];
        }
    }

    // per-column point sums (FP32) and interval events (compensated)
    float P[CPT][V];
    df D[CPT][V];
    df tot[V];
#pragma unroll
    for (int v = 0; v < V; v++) tot[v] = df_zero();
#pragma unroll
    for (int q = 0; q < CPT; q++) {
#pragma unroll
        for (int v = 0; v < V; v++) {
            P[q][v] = 0.f;
            D[q][v] = df_zero();
        }
        const int64_t j = c0 + q;
        if (j < end) {
            const uint32_t e1 = __ldg(colp + j + 1);
            for (uint32_t e = __ldg(colp + j); e < e1; e++) {
                const uint32_t w = __ldg(tent + e);
                Vec<V> zv = ldv<V>(z + (int64_t)id_of(w) * ldz + lane * V);
                const uint32_t tag = w >> kIdBits;
                if (tag < 2) {
#pragma unroll
                    for (int v = 0; v < V; v++) P[q][v] += (tag & 1) ? -zv.v[v] : zv.v[v];
                } else {
#pragma unroll
                    for (int v = 0; v < V; v++) D[q][v] = df_addf(D[q][v], (tag & 1) ? -zv.v[v] : zv.v[v]);
                }
            }
        }
#pragma unroll
        for (int v = 0; v < V; v++) tot[v] = df_add(tot[v], D[q][v]);
    }
    // exclusive prefix of the group totals across the block (compensated)
    df inc[V], ex[V];
#pragma unroll
    for (int v = 0; v < V; v++) inc[v] = tot[v];
#pragma unroll
    for (int d = G; d < 32; d <<= 1)
#pragma unroll
        for (int v = 0; v < V; v++) {
            df o = df_shfl_up(inc[v], d);
            if (lane32 >= d) inc[v] = df_add(o, inc[v]);
        }
#pragma unroll
    for (int v = 0; v < V; v++) {
        df o = df_shfl_up(inc[v], G);
        ex[v] = lane32 >= G ? o : df_zero();
    }
    if (lane32 >= 32 - G) {
#pragma unroll
        for (int v = 0; v < V; v++) wtot_s[warp][lane * V + v] = inc[v];
    }
    __syncthreads();
    df run[V];
#pragma unroll
    for (int v = 0; v < V; v++) {
        df r = run_s[lane * V + v];
        for (int w = 0; w < warp; w++) r = df_add(r, wtot_s[w][lane * V + v]);
        run[v] = df_add(r, ex[v]);
    }

    double S[V], R[V], Dg[V];
#pragma unroll
    for (int v = 0; v < V; v++) S[v] = R[v] = Dg[v] = 0.0;
#pragma unroll
    for (int q = 0; q < CPT; q++) {
        const int64_t j = c0 + q;
        Vec<V> out;
#pragma unroll
        for (int v = 0; v < V; v++) {
            run[v] = df_add(run[v], D[q][v]);
            out.v[v] = df_val(df_addf(run[v], P[q][v]));
        }
        if (j >= end) continue;
        if constexpr (EPI == 0) {
            stv<V>(y + j * ldy + lane * V, out);
        } else {
            const float io = __ldg(pa.inv_outdeg + j);
            const float un = 1.0f / (float)n;
            Vec<V> qp = ldv<V>(pa.q_prev + j * pa.ldq + lane * V), qn, p0v;
            if (pa.p0) p0v = ldv<V>(pa.p0 + j * pa.ldp0 + lane * V);
#pragma unroll
            for (int v = 0; v < V; v++) {
                const float p0j = pa.p0 ? p0v.v[v] : un;
                const float gj = pa.dangling_uniform ? un : p0j;
                const float dl = (float)pa.sc_prev[1 * KB + lane * V + v];
                const float qj = pa.alpha * p0j + (1.0f - pa.alpha) * (out.v[v] + dl * gj);
                qn.v[v] = qj;
                S[v] += (double)qj;
                R[v] += fabs((double)qj - (double)qp.v[v]);
                if (io == 0.0f) Dg[v] += (double)qj;
            }
            stv<V>(pa.q_new + j * pa.ldq + lane * V, qn);
        }
    }
    if constexpr (EPI == 1) pr_block_reduce<KB, V>(S, R, Dg, pa, false);
}

// ---------------------------------------------------------------------------
// y = x A in ONE launch for KB <= 4 right-hand sides (push: Proposition 1 read
// for the left product, then the scatter written as a per-column gather).
//  - Chain step on the fly: the pushed weight of a source row k is
//    z_k = x_k + sum of x over its descendants (desc[k] bit t = row k+t+1),
//    added in increasing row order into a compensated (hi, lo) sum.
//  - Scatter step: y_j = sum_k z_k A'_kj over the column-major entries of the
//    CTA's T columns: points +-z_k (residual/dropped id j of row k) and
//    interval events (start at j: +z_k, end before j: -z_k) whose running
//    prefix is the interval part; the prefix starts from the intervals open
//    at the tile start (carry list), so no grid-wide scan is needed.
//  - Exact accumulation: every term is turned into a 64-bit fixed-point
//    integer with a power-of-two scale chosen per CTA from its own max |z| and
//    term count, so no partial sum overflows; integer sums are exact and
//    associative. The entries are processed EPT consecutive ones per thread
//    (balanced, coalesced); two exclusive prefix sums over this flat stream,
//    C (all terms) and Bp (point terms), are recorded at every column
//    boundary b_j = colp[j], and y_j = carry + C(b_{j+1}) - Bp(b_j): the
//    events of columns <= j plus the points of column j, converted back to
//    FP32 with one rounding. The result is bit-reproducible.
// EPI = 0: store y. EPI = 1: PageRank update (see PrArgs): also writes the
// next iterate q and its pushed input q / outdeg.
// ---------------------------------------------------------------------------
template <int KB>
struct FlatShape {
    static constexpr int NT = 256;
    static constexpr int EPT = 8 / KB;      // entries per thread and chunk
    static constexpr int CE = NT * EPT;     // entries per chunk
    static constexpr int T = 512 / KB;      // columns per CTA
    static constexpr int CPT = (T + NT - 1) / NT;  // columns per thread in the output phase
};

// Scale exponent s with maxabs * terms * 2^s <= 2^62 (maxabs given as float
// bits); integer exponent arithmetic only.
__device__ __forceinline__ int fx_exponent(unsigned int maxbits, long long terms) {
    if (maxbits == 0) return 0;
    const int e_m = (int)((maxbits >> 23) & 0xff) - 126;  // maxabs < 2^e_m
    const int e_t = 64 - __clzll((unsigned long long)terms);  // terms < 2^e_t
    int sexp = 62 - e_m - e_t;
    return sexp > 100 ? 100 : (sexp < -100 ? -100 : sexp);
}

__device__ __forceinline__ float pow2f(int e) {  // 2^e for |e| <= 126
    return __int_as_float((e + 127) << 23);
}

__device__ __forceinline__ long long to_fx(float v, int sexp) {
    // v * 2^s is exact (a power-of-two scaling in range); one rounding to integer
    const float s1 = pow2f(sexp / 2), s2 = pow2f(sexp - sexp / 2);
    return __float2ll_rn(__fmul_rn(__fmul_rn(v, s1), s2));
}

__device__ __forceinline__ float from_fx(long long v, int sexp) {
    const float s1 = pow2f(-(sexp / 2)), s2 = pow2f(-(sexp - sexp / 2));
    return __fmul_rn(__fmul_rn(__ll2float_rn(v), s1), s2);
}

template <int KB>
__device__ __forceinline__ void subtree_sum(const uint32_t* __restrict__ desc, const float* __restrict__ x,
                                            int64_t ldx, uint32_t k, float (&zo)[KB]) {
    Vec<KB> xv = ldv<KB>(x + (int64_t)k * ldx);
    df acc[KB];
#pragma unroll
    for (int v = 0; v < KB; v++) acc[v] = {xv.v[v], 0.f};
    for (uint32_t m = __ldg(desc + k); m; m &= m - 1) {
        Vec<KB> cv = ldv<KB>(x + (int64_t)(k + __ffs(m)) * ldx);
#pragma unroll
        for (int v = 0; v < KB; v++) acc[v] = df_addf(acc[v], cv.v[v]);
    }
#pragma unroll
    for (int v = 0; v < KB; v++) zo[v] = df_val(acc[v]);
}

template <int KB, int EPI>
__global__ void __launch_bounds__(256) k_xA_fused(const uint32_t* __restrict__ colp, const uint32_t* __restrict__ tent,
                                                  const uint32_t* __restrict__ carry_ptr,
                                                  const uint32_t* __restrict__ carry, const uint32_t* __restrict__ desc,
                                                  const float* __restrict__ x, int64_t ldx, float* __restrict__ y,
                                                  int64_t ldy, int64_t n, PrArgs pa) {
    using Sh = FlatShape<KB>;
    constexpr int NT = Sh::NT, EPT = Sh::EPT, CE = Sh::CE, T = Sh::T, CPT = Sh::CPT, NW = NT / 32;
    static_assert(T % kCarryTile == 0, "tile must align with the carry lists");
    if constexpr (EPI == 1) {
        if (__ldcg(&pa.st->done) || __ldcg(&pa.st->iter) >= __ldcg(&pa.st->max_iter)) return;
    }
    __shared__ uint32_t cp_s[T + 1];
    __shared__ uint32_t ent_s[CE + NT];     // skewed: entry e at e + e / EPT
    __shared__ long long cb_s[T + 1][KB];   // C at each column boundary
    __shared__ long long bb_s[T + 1][KB];   // Bp at each column boundary
    __shared__ df run0_s[KB];
    __shared__ long long wtot_s[NW][2][KB];
    __shared__ unsigned int wmax_s[NW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t a = (int64_t)blockIdx.x * T;
    const int ncols = (int)((a + T < n ? a + T : n) - a);
    const int64_t ct = a / kCarryTile;

    for (int i = tid; i <= ncols; i += NT) {
        cp_s[i] = __ldg(colp + a + i);
#pragma unroll
        for (int v = 0; v < KB; v++) cb_s[i][v] = bb_s[i][v] = 0;
    }
    const uint32_t cr0 = __ldg(carry_ptr + ct), cr1 = __ldg(carry_ptr + ct + 1);
    unsigned int mx = 0;  // max |term| as float bits (NaN ranks above every finite value)
    if (warp == 0) {  // running interval prefix at column a (compensated)
        df acc[KB];
#pragma unroll
        for (int v = 0; v < KB; v++) acc[v] = df_zero();
        for (uint32_t e = cr0 + lane; e < cr1; e += 32) {
            float zc[KB];
            subtree_sum<KB>(desc, x, ldx, __ldg(carry + e), zc);
#pragma unroll
            for (int v = 0; v < KB; v++) acc[v] = df_addf(acc[v], zc[v]);
        }
#pragma unroll
        for (int v = 0; v < KB; v++) {
            for (int o = 16; o > 0; o >>= 1)
                acc[v] = df_add(acc[v], {__shfl_down_sync(0xffffffffu, acc[v].hi, o),
                                         __shfl_down_sync(0xffffffffu, acc[v].lo, o)});
            if (lane == 0) {
                run0_s[v] = acc[v];
                mx = max(mx, __float_as_uint(acc[v].hi) & 0x7fffffffu);
            }
        }
    }
    __syncthreads();
    const uint32_t ebase = cp_s[0];
    const int64_t E = (int64_t)cp_s[ncols] - ebase;
    const int nch = (int)((E + CE - 1) / CE);
    const int lo = tid * EPT;

    // terms of this thread for one chunk: z of the source row, signed
    float zf[EPT][KB];
    unsigned int pmask = 0;
    int cnt = 0;
    auto load_chunk = [&](int c) {
        const int64_t cs = (int64_t)c * CE;
        const int ce = (int)(E - cs < CE ? E - cs : CE);
        for (int e = tid; e < ce; e += NT) ent_s[e + e / EPT] = __ldg(tent + ebase + cs + e);
        __syncthreads();
        cnt = ce - lo < 0 ? 0 : (ce - lo > EPT ? EPT : ce - lo);
        // The loads are issued level by level for all EPT entries at once
        // (entry -> source row's mask and x -> first two descendants), so
        // their latencies overlap; rows with more descendants finish in a
        // short loop.
        uint32_t k[EPT], dm[EPT];
        unsigned int neg = 0;
        pmask = 0;
#pragma unroll
        for (int i = 0; i < EPT; i++) {
            const uint32_t w = i < cnt ? ent_s[lo + i + tid] : 0u;
            k[i] = id_of(w);
            if (i < cnt && (w >> kIdBits) < 2) pmask |= 1u << i;
            if ((w >> kIdBits) & 1) neg |= 1u << i;
        }
        Vec<KB> x0[EPT], x1[EPT], x2[EPT];
#pragma unroll
        for (int i = 0; i < EPT; i++) {
            dm[i] = i < cnt ? __ldg(desc + k[i]) : 0u;
            if (i < cnt) x0[i] = ldv<KB>(x + (int64_t)k[i] * ldx);
        }
#pragma unroll
        for (int i = 0; i < EPT; i++) {
            const uint32_t m1 = dm[i], m2 = m1 & (m1 - 1);
#pragma unroll
            for (int v = 0; v < KB; v++) x1[i].v[v] = x2[i].v[v] = 0.f;
            if (m1) x1[i] = ldv<KB>(x + (int64_t)(k[i] + __ffs(m1)) * ldx);
            if (m2) x2[i] = ldv<KB>(x + (int64_t)(k[i] + __ffs(m2)) * ldx);
        }
#pragma unroll
        for (int i = 0; i < EPT; i++) {
            df acc[KB];
#pragma unroll
            for (int v = 0; v < KB; v++) {
                acc[v] = {i < cnt ? x0[i].v[v] : 0.f, 0.f};
                acc[v] = df_addf(df_addf(acc[v], x1[i].v[v]), x2[i].v[v]);
            }
            uint32_t m = dm[i] & (dm[i] - 1);
            m &= m - 1;  // the first two descendants are in
            for (; m; m &= m - 1) {
                Vec<KB> cv = ldv<KB>(x + (int64_t)(k[i] + __ffs(m)) * ldx);
#pragma unroll
                for (int v = 0; v < KB; v++) acc[v] = df_addf(acc[v], cv.v[v]);
            }
#pragma unroll
            for (int v = 0; v < KB; v++) {
                const float zv = df_val(acc[v]);
                zf[i][v] = (neg >> i & 1) ? -zv : zv;
                mx = max(mx, __float_as_uint(zf[i][v]) & 0x7fffffffu);
            }
        }
    };
    // pass 1: the terms (kept in registers when the tile is one chunk) and max |term|
    for (int c = 0; c < nch; c++) {
        if (c > 0) __syncthreads();
        load_chunk(c);
    }
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) wmax_s[warp] = mx;
    __syncthreads();
#pragma unroll
    for (int w2 = 0; w2 < NW; w2++) mx = max(mx, wmax_s[w2]);
    const bool bad = mx >= 0x7f800000u;  // a non-finite term: the product is not defined
    const int sexp = fx_exponent(bad ? 0u : mx, E + 2);
    long long run0[KB];
#pragma unroll
    for (int v = 0; v < KB; v++) run0[v] = to_fx(run0_s[v].hi, sexp) + to_fx(run0_s[v].lo, sexp);

    // pass 2: exact prefix sums, recorded at the column boundaries
    long long chC[KB], chB[KB];
#pragma unroll
    for (int v = 0; v < KB; v++) chC[v] = chB[v] = 0;
    for (int c = 0; c < nch; c++) {
        if (nch > 1) {  // the terms of chunk c are computed again
            __syncthreads();
            load_chunk(c);
        }
        long long tC[KB], tB[KB];
#pragma unroll
        for (int v = 0; v < KB; v++) tC[v] = tB[v] = 0;
#pragma unroll
        for (int i = 0; i < EPT; i++)
#pragma unroll
            for (int v = 0; v < KB; v++) {
                const long long f = to_fx(zf[i][v], sexp);
                tC[v] += f;
                if (pmask >> i & 1) tB[v] += f;
            }
        long long xC[KB], xB[KB], bC[KB], bB[KB];
#pragma unroll
        for (int v = 0; v < KB; v++) {
            long long ic = tC[v], ib = tB[v];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const long long oc = __shfl_up_sync(0xffffffffu, ic, d), ob = __shfl_up_sync(0xffffffffu, ib, d);
                if (lane >= d) {
                    ic += oc;
                    ib += ob;
                }
            }
            if (lane == 31) {
                wtot_s[warp][0][v] = ic;
                wtot_s[warp][1][v] = ib;
            }
            xC[v] = ic - tC[v];
            xB[v] = ib - tB[v];
        }
        __syncthreads();
#pragma unroll
        for (int v = 0; v < KB; v++) {
            bC[v] = bB[v] = 0;
#pragma unroll
            for (int w2 = 0; w2 < NW; w2++) {
                if (w2 < warp) {
                    xC[v] += wtot_s[w2][0][v];
                    xB[v] += wtot_s[w2][1][v];
                }
                bC[v] += wtot_s[w2][0][v];
                bB[v] += wtot_s[w2][1][v];
            }
        }
        if (cnt > 0) {
            const uint32_t first = ebase + (uint32_t)((int64_t)c * CE + lo);  // boundaries b > first
            int j0 = 0, j1 = ncols + 1;
            while (j0 < j1) {  // first j with cp_s[j] > first
                const int mid = (j0 + j1) >> 1;
                if (cp_s[mid] > first) j1 = mid;
                else j0 = mid + 1;
            }
            int j = j0;
            long long rc[KB], rb[KB];
#pragma unroll
            for (int v = 0; v < KB; v++) {
                rc[v] = chC[v] + xC[v];
                rb[v] = chB[v] + xB[v];
            }
#pragma unroll
            for (int i = 0; i < EPT; i++) {
                if (i < cnt) {
#pragma unroll
                    for (int v = 0; v < KB; v++) {
                        const long long f = to_fx(zf[i][v], sexp);
                        rc[v] += f;
                        if (pmask >> i & 1) rb[v] += f;
                    }
                    const uint32_t pos = first + (uint32_t)(i + 1);
                    while (j <= ncols && cp_s[j] == pos) {
#pragma unroll
                        for (int v = 0; v < KB; v++) {
                            cb_s[j][v] = rc[v];
                            bb_s[j][v] = rb[v];
                        }
                        j++;
                    }
                }
            }
        }
#pragma unroll
        for (int v = 0; v < KB; v++) {
            chC[v] += bC[v];
            chB[v] += bB[v];
        }
    }
    __syncthreads();

    double S[KB], R[KB], Dg[KB];
#pragma unroll
    for (int v = 0; v < KB; v++) S[v] = R[v] = Dg[v] = 0.0;
#pragma unroll
    for (int q = 0; q < CPT; q++) {
        const int jl = q * NT + tid;  // consecutive threads, consecutive columns
        if (jl >= ncols) continue;
        const int64_t j = a + jl;
        Vec<KB> out;
#pragma unroll
        for (int v = 0; v < KB; v++)
            out.v[v] = bad ? __int_as_float(0x7fc00000) : from_fx(run0[v] + cb_s[jl + 1][v] - bb_s[jl][v], sexp);
        if constexpr (EPI == 0) {
            stv<KB>(y + j * ldy, out);
        } else {
            const float io = __ldg(pa.inv_outdeg + j);
            const float un = 1.0f / (float)n;
            Vec<KB> qp = ldv<KB>(pa.q_prev + j * pa.ldq), qn, xn, p0v;
            if (pa.p0) p0v = ldv<KB>(pa.p0 + j * pa.ldp0);
#pragma unroll
            for (int v = 0; v < KB; v++) {
                const float p0j = pa.p0 ? p0v.v[v] : un;
                const float gj = pa.dangling_uniform ? un : p0j;
                const float dl = (float)pa.sc_prev[1 * KB + v];
                const float qj = pa.alpha * p0j + (1.0f - pa.alpha) * (out.v[v] + dl * gj);
                qn.v[v] = qj;
                xn.v[v] = __fmul_rn(qj, io);
                S[v] += (double)qj;
                R[v] += fabs((double)qj - (double)qp.v[v]);
                if (io == 0.0f) Dg[v] += (double)qj;
            }
            stv<KB>(pa.q_new + j * pa.ldq, qn);
            stv<KB>(pa.x_new + j * pa.ldq, xn);
        }
    }
    if constexpr (EPI == 1) pr_block_reduce<KB, KB>(S, R, Dg, pa, false);
}

// PageRank start: q_0 = p_init (or p0, or uniform), and the scalars of the
// start (1/S_0, dangling mass) by the same deterministic reduction.
template <int KB, int V>
__global__ void __launch_bounds__(256) k_pr_init(const float* __restrict__ p_init, int64_t ldi, int64_t n,
                                                 int tile, PrArgs pa) {
    constexpr int G = KB / V;
    const int NG = blockDim.x / G;
    const int g = threadIdx.x / G, lane = threadIdx.x % G;
    const int64_t a = (int64_t)blockIdx.x * tile;
    const int64_t end = a + tile < n ? a + tile : n;
    double S[V], R[V], Dg[V];
#pragma unroll
    for (int v = 0; v < V; v++) S[v] = R[v] = Dg[v] = 0.0;
    const float un = 1.0f / (float)n;
    for (int64_t j = a + g; j < end; j += NG) {
        Vec<V> pv;
        if (p_init) pv = ldv<V>(p_init + j * ldi + lane * V);
        else {
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
            S[v] += (double)pv.v[v];
            if (io == 0.0f) Dg[v] += (double)pv.v[v];
        }
    }
    pr_block_reduce<KB, V>(S, R, Dg, pa, true);
}

// p_out = q_T / S_T for the final update T (read from the state).
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
    for (int64_t j = gid; j < n; j += stride) {
        Vec<V> qv = ldv_cg<V>(q + j * ldq + lane * V), o;
#pragma unroll
        for (int v = 0; v < V; v++) o.v[v] = (float)((double)qv.v[v] * __ldcg(sc + lane * V + v));
        stv<V>(out + j * ldo + lane * V, o);
    }
}

}  // namespace bvg

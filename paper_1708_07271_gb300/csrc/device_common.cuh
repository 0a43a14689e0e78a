// Device helpers shared by the kernels: compensated (double-float) FP32
// arithmetic, V-wide vector loads/stores, and launch error plumbing.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "bvg_internal.h"

namespace bvg {

// A value carried as an unevaluated sum hi + lo of two floats. Additions use
// the error-free transformation two_sum (Knuth) on the leading parts and add
// the exact error terms into lo in plain FP32, without renormalising after
// every step: the cascaded summation of Ogita, Rump and Oishi ("Sum2",
// Accurate sum and dot product, 2005), whose result hi + lo is as accurate as
// if computed in twice the working precision and then rounded (error at most
// eps |s| + gamma_{n-1}^2 sum |x_i| for n terms). A chain of additions thus
// loses about one FP32 rounding in total instead of one per addition.
struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_zero() { return {0.f, 0.f}; }

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// a + b for two compensated values (cascaded: the error terms accumulate in lo).
__device__ __forceinline__ df df_add(df a, df b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    return {s, __fadd_rn(e, __fadd_rn(a.lo, b.lo))};
}

// a + b with the result renormalised (|lo| <= ulp(hi) / 2): for long running
// sums with cancellation (prefixes of +/- events), where the unnormalised
// form's second-order error term (n eps)^2 sum |x| is not negligible.
__device__ __forceinline__ df df_add_rn(df a, df b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float h = __fadd_rn(s, e);
    return {h, __fsub_rn(e, __fsub_rn(h, s))};
}

// a + b for a compensated value and a float.
__device__ __forceinline__ df df_addf(df a, float b) {
    float s, e;
    two_sum(a.hi, b, s, e);
    return {s, __fadd_rn(a.lo, e)};
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ float df_val(df a) { return __fadd_rn(a.hi, a.lo); }

__device__ __forceinline__ df df_shfl_xor(df v, int d) {
    return {__shfl_xor_sync(0xffffffffu, v.hi, d), __shfl_xor_sync(0xffffffffu, v.lo, d)};
}

__device__ __forceinline__ df df_shfl_up(df v, int d) {
    return {__shfl_up_sync(0xffffffffu, v.hi, d), __shfl_up_sync(0xffffffffu, v.lo, d)};
}

// V consecutive floats (V in {1, 2, 4}); the caller guarantees alignment.
template <int V>
struct Vec {
    float v[V];
};

template <int V>
__device__ __forceinline__ Vec<V> ldv(const float* p) {
    Vec<V> r;
    if constexpr (V == 4) {
        float4 t = __ldg(reinterpret_cast<const float4*>(p));
        r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
    } else if constexpr (V == 2) {
        float2 t = __ldg(reinterpret_cast<const float2*>(p));
        r.v[0] = t.x; r.v[1] = t.y;
    } else {
        r.v[0] = __ldg(p);
    }
    return r;
}

// Load through L2 only (data written earlier in the same kernel sequence
// by other CTAs must not be served from a stale L1 line).
template <int V>
__device__ __forceinline__ Vec<V> ldv_cg(const float* p) {
    Vec<V> r;
    if constexpr (V == 4) {
        float4 t = __ldcg(reinterpret_cast<const float4*>(p));
        r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
    } else if constexpr (V == 2) {
        float2 t = __ldcg(reinterpret_cast<const float2*>(p));
        r.v[0] = t.x; r.v[1] = t.y;
    } else {
        r.v[0] = __ldcg(p);
    }
    return r;
}

// Coherent load cached in L1 (ld.global.ca): for data written by the
// previous kernel when this kernel may start before that kernel ends
// (programmatic dependent launch) -- read only after griddepcontrol.wait.
template <int V>
__device__ __forceinline__ Vec<V> ldv_ca(const float* p) {
    Vec<V> r;
    if constexpr (V == 4) {
        float4 t = __ldca(reinterpret_cast<const float4*>(p));
        r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
    } else if constexpr (V == 2) {
        float2 t = __ldca(reinterpret_cast<const float2*>(p));
        r.v[0] = t.x; r.v[1] = t.y;
    } else {
        r.v[0] = __ldca(p);
    }
    return r;
}

template <int V>
__device__ __forceinline__ void stv(float* p, const Vec<V>& r) {
    if constexpr (V == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
    } else if constexpr (V == 2) {
        *reinterpret_cast<float2*>(p) = make_float2(r.v[0], r.v[1]);
    } else {
        *p = r.v[0];
    }
}

__device__ __forceinline__ uint32_t tag_of(uint32_t w) { return w >> kIdBits; }
__device__ __forceinline__ uint32_t id_of(uint32_t w) { return w & kIdMask; }

}  // namespace bvg

// Host-side: turn a CUDA error into a library status.
#define BVG_CUDA_TRY(expr)                                                                       \
    do {                                                                                         \
        cudaError_t e_ = (expr);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            cudaGetLastError(); /* do not leave a non-sticky error for the caller's next check */ \
            return ::bvg::fail(BVG_ERR_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                               __LINE__);                                                        \
        }                                                                                        \
    } while (0)

// Learned warm start for PageRank: node features, a 6 -> 64 -> 64 -> 1 ReLU
// network (BF16 weights, FP32 accumulation; the 64 x 64 layer on tensor
// cores with mma.sync m16n8k16), its backward pass and Adam, and the warm
// start p_init ~ max(prediction, floor). The network predicts n p*_i (the
// PageRank vector scaled to mean 1). The power iteration (Eq. 1) converges
// to the same fixed point from any start; a better start only saves updates.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "kernels.cuh"

using namespace bvg;

namespace bvg {

constexpr int MH = 64, MF = 6, FSTR = 8;
constexpr int OFF_W1 = 0, OFF_B1 = MH * MF, OFF_W2 = OFF_B1 + MH, OFF_B2 = OFF_W2 + MH * MH, OFF_W3 = OFF_B2 + MH,
              OFF_B3 = OFF_W3 + MH, NPARAM = OFF_B3 + 1;
constexpr int QW1 = 0, QW2 = MH * MF, QW3 = QW2 + MH * MH, NQ = QW3 + MH;  // bf16 copies of W1, W2, w3
constexpr int MT = 128;  // nodes per CTA (4 warps x 32)
constexpr int HP = 72;   // padded bf16 row of H1 / W2 in shared memory
constexpr int FP = 65;   // padded f32 row of H2 / dH2 / dH1

struct MlpSmem {
    float w1[MH * MF];
    float b1[MH], b2[MH], w3[MH];
    float b3;
    float dy[MT];
    __nv_bfloat16 w2[MH * HP];
    __nv_bfloat16 h1[MT * HP];
};
struct MlpSmemTrain {
    float f[MT * MF];
    float w2f[MH * MH];
    float h2[MT * FP];
    float dh2[MT * FP];
    float dh1[MT * FP];
};

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// Forward (and with TRAIN the backward) of one CTA of MT nodes.
//   a1 = W1q f + b1, h1q = bf16(relu(a1)); a2 = W2q h1q + b2 (tensor cores),
//   h2 = relu(a2); yhat = w3q . h2 + b3.
// TRAIN: dy = 2 (yhat - t) / norm_n; gradients of the mean squared error
// accumulate into grad (atomics across CTAs), the loss sum into *loss.
template <bool TRAIN>
__global__ void __launch_bounds__(MT) k_mlp(const float* __restrict__ feat, const float* __restrict__ target,
                                            int64_t n, double norm_n, const float* __restrict__ theta,
                                            const __nv_bfloat16* __restrict__ wq, float* __restrict__ out,
                                            float* __restrict__ grad, double* __restrict__ loss) {
    extern __shared__ float4 mlp_dyn_smem[];
    MlpSmem& S = *reinterpret_cast<MlpSmem*>(mlp_dyn_smem);
    MlpSmemTrain& U = *reinterpret_cast<MlpSmemTrain*>(reinterpret_cast<char*>(mlp_dyn_smem) + sizeof(MlpSmem));
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, gid = lane >> 2, tig = lane & 3;
    const int64_t base = (int64_t)blockIdx.x * MT, node = base + t;
    const bool valid = node < n;

    for (int i = t; i < MH * MF; i += MT) S.w1[i] = __bfloat162float(wq[QW1 + i]);
    for (int i = t; i < MH; i += MT) {
        S.b1[i] = theta[OFF_B1 + i];
        S.b2[i] = theta[OFF_B2 + i];
        S.w3[i] = __bfloat162float(wq[QW3 + i]);
    }
    if (t == 0) S.b3 = theta[OFF_B3];
    for (int i = t; i < MH * MH; i += MT) {
        S.w2[(i / MH) * HP + i % MH] = wq[QW2 + i];
        if constexpr (TRAIN) U.w2f[i] = __bfloat162float(wq[QW2 + i]);
    }
    float f[MF];
    {
        float4 f0 = make_float4(0.f, 0.f, 0.f, 0.f), f1 = f0;
        if (valid) {
            f0 = __ldg(reinterpret_cast<const float4*>(feat + node * FSTR));
            f1 = __ldg(reinterpret_cast<const float4*>(feat + node * FSTR + 4));
        }
        f[0] = f0.x; f[1] = f0.y; f[2] = f0.z; f[3] = f0.w; f[4] = f1.x; f[5] = f1.y;
    }
    if constexpr (TRAIN)
#pragma unroll
        for (int i = 0; i < MF; i++) U.f[t * MF + i] = valid ? f[i] : 0.f;
    __syncthreads();
    // layer 1 (CUDA cores)
    for (int o = 0; o < MH; o++) {
        float a = S.b1[o];
#pragma unroll
        for (int i = 0; i < MF; i++) a = fmaf(S.w1[o * MF + i], f[i], a);
        S.h1[t * HP + o] = __float2bfloat16_rn(valid ? fmaxf(a, 0.f) : 0.f);
    }
    __syncthreads();
    // layer 2 (tensor cores): warp w computes rows [32w, 32w + 32) x 64 columns
    float acc[2][8][4];
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int nt = 0; nt < 8; nt++)
#pragma unroll
            for (int e = 0; e < 4; e++) acc[mt][nt][e] = 0.f;
#pragma unroll
    for (int ks = 0; ks < 4; ks++) {
        const int k0 = ks * 16 + 2 * tig;
#pragma unroll
        for (int mt = 0; mt < 2; mt++) {
            const int r0 = warp * 32 + mt * 16 + gid;
            const uint32_t a0 = ld32(&S.h1[r0 * HP + k0]), a1 = ld32(&S.h1[(r0 + 8) * HP + k0]);
            const uint32_t a2 = ld32(&S.h1[r0 * HP + k0 + 8]), a3 = ld32(&S.h1[(r0 + 8) * HP + k0 + 8]);
#pragma unroll
            for (int nt = 0; nt < 8; nt++) {
                const int nrow = nt * 8 + gid;
                mma_bf16(acc[mt][nt], a0, a1, a2, a3, ld32(&S.w2[nrow * HP + k0]), ld32(&S.w2[nrow * HP + k0 + 8]));
            }
        }
    }
    // bias, ReLU, output layer
    float yp[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int nt = 0; nt < 8; nt++)
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int col = nt * 8 + 2 * tig + (e & 1), half = e >> 1;
                const int row = warp * 32 + mt * 16 + gid + 8 * half;
                const float h2 = fmaxf(acc[mt][nt][e] + S.b2[col], 0.f);
                yp[mt][half] = fmaf(S.w3[col], h2, yp[mt][half]);
                if constexpr (TRAIN) U.h2[row * FP + col] = h2;
            }
    double lsum = 0.0;
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int half = 0; half < 2; half++) {
            float y = yp[mt][half];
            y += __shfl_xor_sync(0xffffffffu, y, 1);
            y += __shfl_xor_sync(0xffffffffu, y, 2);
            y += S.b3;
            const int row = warp * 32 + mt * 16 + gid + 8 * half;
            const int64_t nd = base + row;
            if (tig == 0) {
                if (out && nd < n) out[nd] = y;
                if constexpr (TRAIN) {
                    const float r = nd < n ? y - __ldg(target + nd) : 0.f;
                    S.dy[row] = (float)(2.0 * (double)r / norm_n);
                    lsum += (double)r * (double)r;
                }
            }
        }
    if constexpr (TRAIN) {
        for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
        if (lane == 0) atomicAdd(loss, lsum);
        __syncthreads();
        // dh2 = dy w3q [a2 > 0]
        for (int c = 0; c < MH; c++) U.dh2[t * FP + c] = U.h2[t * FP + c] > 0.f ? S.dy[t] * S.w3[c] : 0.f;
        __syncthreads();
        // gradients of W2 (dh2^T h1q), b2, w3, b3
        for (int o = t; o < MH * MH; o += MT) {
            const int nn = o / MH, k = o % MH;
            float g = 0.f;
            for (int r = 0; r < MT; r++) g = fmaf(U.dh2[r * FP + nn], __bfloat162float(S.h1[r * HP + k]), g);
            atomicAdd(grad + OFF_W2 + o, g);
        }
        if (t < MH) {
            float gb = 0.f, gw = 0.f;
            for (int r = 0; r < MT; r++) {
                gb += U.dh2[r * FP + t];
                gw = fmaf(S.dy[r], U.h2[r * FP + t], gw);
            }
            atomicAdd(grad + OFF_B2 + t, gb);
            atomicAdd(grad + OFF_W3 + t, gw);
        } else if (t == MH) {
            float gb = 0.f;
            for (int r = 0; r < MT; r++) gb += S.dy[r];
            atomicAdd(grad + OFF_B3, gb);
        }
        // dh1 = W2q^T dh2 [a1 > 0]
        for (int k = 0; k < MH; k++) {
            float s = 0.f;
            for (int c = 0; c < MH; c++) s = fmaf(U.w2f[c * MH + k], U.dh2[t * FP + c], s);
            U.dh1[t * FP + k] = __bfloat162float(S.h1[t * HP + k]) > 0.f ? s : 0.f;
        }
        __syncthreads();
        // gradients of W1 (dh1^T f) and b1
        for (int o = t; o < MH * MF; o += MT) {
            const int oo = o / MF, i = o % MF;
            float g = 0.f;
            for (int r = 0; r < MT; r++) g = fmaf(U.dh1[r * FP + oo], U.f[r * MF + i], g);
            atomicAdd(grad + OFF_W1 + o, g);
        }
        if (t < MH) {
            float g = 0.f;
            for (int r = 0; r < MT; r++) g += U.dh1[r * FP + t];
            atomicAdd(grad + OFF_B1 + t, g);
        }
    }
}

__global__ void k_quantize(const float* __restrict__ theta, __nv_bfloat16* __restrict__ wq) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NQ; i += gridDim.x * blockDim.x) {
        const int src = i < QW2 ? OFF_W1 + i : (i < QW3 ? OFF_W2 + (i - QW2) : OFF_W3 + (i - QW3));
        wq[i] = __float2bfloat16_rn(theta[src]);
    }
}

// Adam (bias-corrected); then the bf16 copies of the weights are refreshed.
__global__ void k_adam(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ grad, float lr, float c1, float c2, float beta1, float beta2,
                       float eps) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NPARAM; i += gridDim.x * blockDim.x) {
        const float g = grad[i];
        const float mi = beta1 * m[i] + (1.f - beta1) * g;
        const float vi = beta2 * v[i] + (1.f - beta2) * g * g;
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

// Node features (stride FSTR): log1p(indeg), log1p(outdeg), chain depth,
// interval members / outdeg, log1p(mean successor out-degree),
// log1p(weighted in-degree). deg holds (indeg, weighted indeg) per node.
__global__ void k_features(const uint8_t* __restrict__ meta, const uint32_t* __restrict__ rowp,
                           const uint32_t* __restrict__ ent, const float* __restrict__ inv_outdeg,
                           const float2* __restrict__ deg, const float* __restrict__ nbrsum, int64_t n,
                           float* __restrict__ feat) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float inv = __ldg(inv_outdeg + i);
        const float od = inv > 0.f ? rintf(1.0f / inv) : 0.f;
        uint32_t members = 0;
        for (uint32_t w = __ldg(rowp + i); w < __ldg(rowp + i + 1); w++) {
            const uint32_t word = __ldg(ent + w);
            if (tag_of(word) == kTagIvL) members += id_of(word);
        }
        const float mean_nbr = od > 0.f ? __ldg(nbrsum + i) / od : 0.f;
        const float2 d = deg[i];
        float4 a = make_float4(log1pf(d.x), log1pf(od), (float)(__ldg(meta + i) >> kMetaDepthShift),
                               od > 0.f ? (float)members / od : 0.f);
        float4 b = make_float4(log1pf(mean_nbr), log1pf(d.y), 0.f, 0.f);
        *reinterpret_cast<float4*>(feat + i * FSTR) = a;
        *reinterpret_cast<float4*>(feat + i * FSTR + 4) = b;
    }
}

// Inputs of the two degree products: x = (1, 1/outdeg) per node (n x 2) for
// 1 A and (1/outdeg) A, and outdeg for A outdeg^T.
__global__ void k_degree_inputs(const float* __restrict__ inv_outdeg, int64_t n, float2* __restrict__ x2,
                                float* __restrict__ od) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float inv = __ldg(inv_outdeg + i);
        x2[i] = make_float2(1.0f, inv);
        od[i] = inv > 0.f ? rintf(1.0f / inv) : 0.f;
    }
}

// Training target t_i = n p*_i.
__global__ void k_targets(const float* __restrict__ p, int64_t n, float* __restrict__ t) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        t[i] = (float)n * __ldg(p + i);
}

// p_i = max(yhat_i, floor) (NaN maps to the floor) and its sum (FP64,
// per-CTA partials in a fixed order).
__global__ void __launch_bounds__(256) k_floor_sum(const float* __restrict__ yhat, int64_t n, float floor_v,
                                                   float* __restrict__ p, double* __restrict__ part) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float e = fmaxf(__ldg(yhat + i), floor_v);  // fmaxf returns floor_v for a NaN prediction
        p[i] = e;
        s += (double)e;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// p /= sum(partials); a non-finite or non-positive sum falls back to 1/n.
// Every CTA adds the partials the same way (its threads strided over them,
// then a fixed tree); each value is scaled by 1/sum rounded once to FP32
// (FP64 division per value would run at the small FP64 rate of this part).
__global__ void __launch_bounds__(256) k_normalize(float* __restrict__ p, int64_t n, const double* __restrict__ part,
                                                   int nparts) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += __ldcg(part + i);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    const double tot = sh[0];
    const bool ok = tot > 0.0 && isfinite(tot);
    const float inv = ok ? (float)(1.0 / tot) : 0.0f, un = 1.0f / (float)n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = ok ? __fmul_rn(p[i], inv) : un;
        p[i] = isfinite(v) ? v : un;
    }
}

constexpr float kWarmFloor = 0.05f;  // lower bound of n p_init (n p*_i >= alpha for uniform teleport)

static size_t mlp_smem(bool train) { return sizeof(MlpSmem) + (train ? sizeof(MlpSmemTrain) : 0); }

}  // namespace bvg

struct bvg_mlp {
    int device = 0;
    float* theta = nullptr;  // FP32 master parameters
    float* m = nullptr;
    float* v = nullptr;
    float* grad = nullptr;
    __nv_bfloat16* wq = nullptr;
    double* loss = nullptr;
    double* part = nullptr;  // exp-sum partials
    int64_t step = 0;
};

namespace bvg {

static int mlp_alloc(void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(BVG_ERR_OOM, "warm-start network: cudaMalloc(%zu) failed", bytes);
    }
    return BVG_OK;
}

static uint64_t sm64(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static int launch_mlp(const bvg_mlp* net, bool train, const float* feat, const float* target, int64_t n,
                      double norm_n, float* out, cudaStream_t st) {
    const size_t smem = mlp_smem(train);
    auto kern = train ? k_mlp<true> : k_mlp<false>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int64_t grid = (n + MT - 1) / MT;
    kern<<<(unsigned)grid, MT, smem, st>>>(feat, target, n, norm_n, net->theta, net->wq, out, net->grad, net->loss);
    BVG_CUDA_TRY(cudaGetLastError());
    return BVG_OK;
}

static int grid_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 16); }

// Features of g into feat (device n x 8).
static int features(const bvg_dev_graph* gc, float* feat, cudaStream_t st) {
    bvg_dev_graph* g = const_cast<bvg_dev_graph*>(gc);
    const int64_t n = g->n;
    if (g->s.feat_cap < n) {
        if (g->s.feat_tmp) cudaFree(g->s.feat_tmp);
        g->s.feat_tmp = nullptr;
        g->s.feat_cap = 0;
        int rc = mlp_alloc((void**)&g->s.feat_tmp, (size_t)n * 6 * sizeof(float));
        if (rc) return rc;
        g->s.feat_cap = n;
    }
    float* x2 = g->s.feat_tmp;  // n x 2
    float* deg = x2 + 2 * n;    // n x 2: in-degree, weighted in-degree
    float* od = deg + 2 * n;
    float* nbr = od + n;
    k_degree_inputs<<<grid_for(n), 256, 0, st>>>(g->inv_outdeg, n, reinterpret_cast<float2*>(x2), od);
    int rc = bvg_spmv_xA(g, x2, deg, 2, 2, st);  // (1, 1/outdeg) A
    if (rc) return rc;
    rc = bvg_spmv_Ax(g, od, nbr, 1, 1, st);  // sum of successor out-degrees: A outdeg
    if (rc) return rc;
    k_features<<<grid_for(n), 256, 0, st>>>(g->meta, g->rowp, g->ent, g->inv_outdeg,
                                            reinterpret_cast<const float2*>(deg), nbr, n, feat);
    BVG_CUDA_TRY(cudaGetLastError());
    return BVG_OK;
}

static int adam_step(bvg_mlp* net, float lr, cudaStream_t st) {
    net->step++;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 / (1.0 - std::pow(b1, (double)net->step)));
    const float c2 = (float)(1.0 / (1.0 - std::pow(b2, (double)net->step)));
    k_adam<<<(NPARAM + 255) / 256, 256, 0, st>>>(net->theta, net->m, net->v, net->grad, lr, c1, c2, (float)b1,
                                                (float)b2, 1e-8f);
    k_quantize<<<(NQ + 255) / 256, 256, 0, st>>>(net->theta, net->wq);
    BVG_CUDA_TRY(cudaGetLastError());
    return BVG_OK;
}

}  // namespace bvg

// ==================================================================== C ABI
extern "C" int bvg_mlp_create(uint64_t seed, bvg_mlp** out) {
    if (!out) return fail(BVG_ERR_INVALID_ARG, "bvg_mlp_create: out is NULL");
    *out = nullptr;
    bvg_mlp* net = new (std::nothrow) bvg_mlp();
    if (!net) return fail(BVG_ERR_OOM, "bvg_mlp_create: host allocation failed");
    int rc;
    BVG_CUDA_TRY(cudaGetDevice(&net->device));
    if ((rc = mlp_alloc((void**)&net->theta, NPARAM * sizeof(float))) ||
        (rc = mlp_alloc((void**)&net->m, NPARAM * sizeof(float))) ||
        (rc = mlp_alloc((void**)&net->v, NPARAM * sizeof(float))) ||
        (rc = mlp_alloc((void**)&net->grad, NPARAM * sizeof(float))) ||
        (rc = mlp_alloc((void**)&net->wq, NQ * sizeof(__nv_bfloat16))) ||
        (rc = mlp_alloc((void**)&net->loss, sizeof(double))) ||
        (rc = mlp_alloc((void**)&net->part, 152 * 16 * sizeof(double)))) {
        bvg_free_mlp(net);
        return rc;
    }
    // He-style initial weights from a splitmix64 stream (Box-Muller), zero biases
    std::vector<float> h(NPARAM, 0.f);
    uint64_t s = seed;
    auto normal = [&]() {
        const double u1 = ((sm64(s) >> 11) + 1.0) * (1.0 / 9007199254740993.0), u2 = (sm64(s) >> 11) * (1.0 / 9007199254740992.0);
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    };
    for (int i = 0; i < MH * MF; i++) h[OFF_W1 + i] = (float)(normal() * std::sqrt(2.0 / MF));
    for (int i = 0; i < MH * MH; i++) h[OFF_W2 + i] = (float)(normal() * std::sqrt(2.0 / MH));
    for (int i = 0; i < MH; i++) h[OFF_W3 + i] = (float)(normal() * std::sqrt(1.0 / MH));
    rc = bvg_mlp_set_params(net, h.data(), NPARAM);
    if (rc) {
        bvg_free_mlp(net);
        return rc;
    }
    *out = net;
    return BVG_OK;
}

extern "C" int bvg_mlp_set_params(bvg_mlp* net, const float* host, int64_t count) {
    if (!net || !host || count != NPARAM)
        return fail(BVG_ERR_INVALID_ARG, "bvg_mlp_set_params: need %d host floats", NPARAM);
    BVG_CUDA_TRY(cudaMemcpy(net->theta, host, NPARAM * sizeof(float), cudaMemcpyHostToDevice));
    BVG_CUDA_TRY(cudaMemset(net->m, 0, NPARAM * sizeof(float)));
    BVG_CUDA_TRY(cudaMemset(net->v, 0, NPARAM * sizeof(float)));
    net->step = 0;
    k_quantize<<<(NQ + 255) / 256, 256>>>(net->theta, net->wq);
    BVG_CUDA_TRY(cudaGetLastError());
    BVG_CUDA_TRY(cudaDeviceSynchronize());
    return BVG_OK;
}

extern "C" int bvg_mlp_get_params(const bvg_mlp* net, float* host, int64_t count) {
    if (!net || !host || count != NPARAM)
        return fail(BVG_ERR_INVALID_ARG, "bvg_mlp_get_params: need %d host floats", NPARAM);
    BVG_CUDA_TRY(cudaDeviceSynchronize());
    BVG_CUDA_TRY(cudaMemcpy(host, net->theta, NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    return BVG_OK;
}

extern "C" int bvg_features(const bvg_dev_graph* g, float* feat, void* stream) {
    if (!g || !feat) return fail(BVG_ERR_INVALID_ARG, "bvg_features: NULL argument");
    if ((uintptr_t)feat % 16) return fail(BVG_ERR_INVALID_ARG, "bvg_features: feat must be 16-byte aligned");
    if (g->n == 0) return BVG_OK;
    return features(g, feat, (cudaStream_t)stream);
}

extern "C" int bvg_mlp_predict(const bvg_mlp* net, const float* feat, int64_t n, float* out, void* stream) {
    if (!net || !feat || !out || n < 0) return fail(BVG_ERR_INVALID_ARG, "bvg_mlp_predict: bad argument");
    if ((uintptr_t)feat % 16) return fail(BVG_ERR_INVALID_ARG, "bvg_mlp_predict: feat must be 16-byte aligned");
    if (n == 0) return BVG_OK;
    return launch_mlp(net, false, feat, nullptr, n, 1.0, out, (cudaStream_t)stream);
}

extern "C" int bvg_mlp_grad(bvg_mlp* net, const float* feat, const float* target, int64_t n, double* loss_out,
                            float* grad_host, void* stream) {
    if (!net || !feat || !target || n <= 0) return fail(BVG_ERR_INVALID_ARG, "bvg_mlp_grad: bad argument");
    if ((uintptr_t)feat % 16) return fail(BVG_ERR_INVALID_ARG, "bvg_mlp_grad: feat must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    BVG_CUDA_TRY(cudaMemsetAsync(net->grad, 0, NPARAM * sizeof(float), st));
    BVG_CUDA_TRY(cudaMemsetAsync(net->loss, 0, sizeof(double), st));
    int rc = launch_mlp(net, true, feat, target, n, (double)n, nullptr, st);
    if (rc) return rc;
    double l = 0;
    BVG_CUDA_TRY(cudaMemcpyAsync(&l, net->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (grad_host) BVG_CUDA_TRY(cudaMemcpyAsync(grad_host, net->grad, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, st));
    BVG_CUDA_TRY(cudaStreamSynchronize(st));
    if (loss_out) *loss_out = l / (double)n;
    return BVG_OK;
}

extern "C" int bvg_mlp_adam(bvg_mlp* net, float lr, void* stream) {
    if (!net || !(lr > 0)) return fail(BVG_ERR_INVALID_ARG, "bvg_mlp_adam: bad argument");
    return adam_step(net, lr, (cudaStream_t)stream);
}

extern "C" int bvg_warmstart_train(bvg_mlp* net, const bvg_dev_graph* const* gs, const float* const* p_star,
                                   int32_t count, int32_t epochs, float lr, int64_t batch, double* loss_out,
                                   void* stream) {
    if (!net || !gs || !p_star || count < 1 || epochs < 1 || !(lr > 0) || batch < MT)
        return fail(BVG_ERR_INVALID_ARG, "bvg_warmstart_train: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<float*> feats(count, nullptr), tgts(count, nullptr);
    int rc = BVG_OK;
    auto cleanup = [&]() {
        for (float* p : feats)
            if (p) cudaFree(p);
        for (float* p : tgts)
            if (p) cudaFree(p);
    };
    for (int gi = 0; gi < count && !rc; gi++) {
        const int64_t n = gs[gi]->n;
        if ((rc = mlp_alloc((void**)&feats[gi], (size_t)std::max<int64_t>(n, 1) * FSTR * sizeof(float))) ||
            (rc = mlp_alloc((void**)&tgts[gi], (size_t)std::max<int64_t>(n, 1) * sizeof(float))))
            break;
        if (n == 0) continue;
        if ((rc = features(gs[gi], feats[gi], st))) break;
        k_targets<<<grid_for(n), 256, 0, st>>>(p_star[gi], n, tgts[gi]);
    }
    double last = 0.0;
    int64_t last_n = 0;
    for (int ep = 0; ep < epochs && !rc; ep++) {
        last = 0.0;
        last_n = 0;
        for (int gi = 0; gi < count && !rc; gi++) {
            const int64_t n = gs[gi]->n;
            for (int64_t c0 = 0; c0 < n && !rc; c0 += batch) {
                const int64_t cn = std::min(batch, n - c0);
                double l = 0.0;
                if ((rc = bvg_mlp_grad(net, feats[gi] + c0 * FSTR, tgts[gi] + c0, cn, &l, nullptr, st))) break;
                rc = adam_step(net, lr, st);
                last += l * (double)cn;
                last_n += cn;
            }
        }
    }
    if (!rc) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = fail(BVG_ERR_CUDA, "bvg_warmstart_train: %s", cudaGetErrorString(e));
    }
    cleanup();
    if (!rc && loss_out) *loss_out = last_n ? last / (double)last_n : 0.0;
    return rc;
}

extern "C" int bvg_warmstart_predict(const bvg_mlp* net, const bvg_dev_graph* g, float* p_init, void* stream) {
    if (!net || !g || !p_init) return fail(BVG_ERR_INVALID_ARG, "bvg_warmstart_predict: NULL argument");
    const int64_t n = g->n;
    if (n == 0) return BVG_OK;
    cudaStream_t st = (cudaStream_t)stream;
    bvg_dev_graph* gm = const_cast<bvg_dev_graph*>(g);
    if (gm->s.wfeat_cap < n) {
        if (gm->s.wfeat) cudaFree(gm->s.wfeat);
        gm->s.wfeat = nullptr;
        gm->s.wfeat_cap = 0;
        int rc = mlp_alloc((void**)&gm->s.wfeat, (size_t)n * (FSTR + 1) * sizeof(float));
        if (rc) return rc;
        gm->s.wfeat_cap = n;
    }
    float* feat = gm->s.wfeat;
    float* yhat = feat + n * FSTR;
    int rc = features(g, feat, st);
    if (rc) return rc;
    if ((rc = launch_mlp(net, false, feat, nullptr, n, 1.0, yhat, st))) return rc;
    const int grid = grid_for(n);
    k_floor_sum<<<grid, 256, 0, st>>>(yhat, n, kWarmFloor, p_init, net->part);
    k_normalize<<<grid, 256, 0, st>>>(p_init, n, net->part, grid);
    BVG_CUDA_TRY(cudaGetLastError());
    return BVG_OK;
}

extern "C" void bvg_free_mlp(bvg_mlp* net) {
    if (!net) return;
    void* ptrs[] = {net->theta, net->m, net->v, net->grad, net->wq, net->loss, net->part};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete net;
}

extern "C" int bvg_mlp_param_count(void) { return NPARAM; }

// y = x A without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need the
// product: code that runs under a memory budget owned by another allocator
// (a framework's caching pool that must see every byte), latency-critical
// loops where cudaMalloc's implicit device synchronisation is not acceptable,
// and embedders that forbid the library from growing its footprint after
// start-up. bvg_spmv_xA may allocate on its first call with a larger k (it
// grows the handle's scratch buffer); this entry point never does. Its
// scratch -- the pushed weights z, n x kb floats -- lives in a fixed
// file-scope device array that every GPU which loads this library holds
// until the process exits.
#include <mutex>

#include "kernels.cuh"

using namespace bvg;

namespace {

// 16 MiB of scratch: n * kb <= 4,194,304 floats.
constexpr int64_t kNoAllocScratchFloats = (int64_t)1 << 22;
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device. In host code
// g_noalloc_scratch names a host-side stand-in, not device memory, so the
// address is looked up once per device (with that device current) and kept.
int scratch_on_current_device(float** out) {
    int dev = 0;
    BVG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(BVG_ERR_UNSUPPORTED, "bvg_spmv_xA_noalloc: device %d", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fail(BVG_ERR_CUDA, "bvg_spmv_xA_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        }
        g_scratch_ptr[dev] = (float*)p;
    }
    *out = g_scratch_ptr[dev];
    return BVG_OK;
}

int pick_v_na(int kb, int64_t ld, int64_t col, const void* x, const void* y) {
    auto ok = [&](int v) {
        if (kb % v || ld % v || col % v) return false;
        for (const void* p : {x, y})
            if (((uintptr_t)((const float*)p + col) % (4 * v))) return false;
        return true;
    };
    if (kb >= 4 && ok(4)) return 4;
    if (kb == 2 && ok(2)) return 2;
    return 1;
}

// The same two kernels as bvg_spmv_xA (chain step, then the per-column
// gather), launched one after the other in plain stream order.
template <int KB, int V>
void launch_pair(const bvg_dev_graph* g, const float* x, int64_t ld, float* z, float* y, cudaStream_t st) {
    const int64_t cgrid = (g->n + ChainShape<KB, V>::TILE - 1) / ChainShape<KB, V>::TILE;
    k_chain<KB, V><<<(unsigned)cgrid, ChainShape<KB, V>::NT, 0, st>>>(g->desc, x, ld, nullptr, z, KB, g->n, nullptr);
    const int64_t ggrid = (g->n + GatherShape<KB, V>::T - 1) / GatherShape<KB, V>::T;
    PrArgs pa{};
    k_gather<KB, V, 0><<<(unsigned)ggrid, GatherShape<KB, V>::NT, 0, st>>>(g->colp, g->tent, g->titem_ptr, g->titem,
                                                                         g->carry_ptr, g->carry,
                                                                         z, KB, y, ld, g->n, pa);
}

}  // namespace

extern "C" int bvg_spmv_xA_noalloc(const bvg_dev_graph* g, const float* x, float* y, int32_t k, int64_t ld,
                                   void* stream) {
    if (!g || !x || !y) return fail(BVG_ERR_INVALID_ARG, "bvg_spmv_xA_noalloc: NULL argument");
    if (k < 1 || ld < k) return fail(BVG_ERR_INVALID_ARG, "bvg_spmv_xA_noalloc: need k >= 1 and ld >= k");
    if (x == y) return fail(BVG_ERR_INVALID_ARG, "bvg_spmv_xA_noalloc: x and y must not alias");
    if (g->n == 0) return BVG_OK;
    // the kernels below run on the current device against the graph's
    // structure arrays and the current device's scratch: both must be the
    // graph's device, and x, y its memory (a host or foreign pointer is
    // refused here rather than faulting in a kernel)
    int cur = -1;
    BVG_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != g->device)
        return fail(BVG_ERR_INVALID_ARG, "bvg_spmv_xA_noalloc: current device %d is not the graph's device %d", cur,
                    g->device);
    int rc0;
    if ((rc0 = check_vec(g, x, "x")) || (rc0 = check_vec(g, y, "y"))) return rc0;
    if (g->n > kNoAllocScratchFloats)
        return fail(BVG_ERR_UNSUPPORTED,
                    "bvg_spmv_xA_noalloc: n = %lld exceeds the fixed scratch of %lld floats (n * column block "
                    "must be <= %lld)",
                    (long long)g->n, (long long)kNoAllocScratchFloats, (long long)kNoAllocScratchFloats);
    float* z = nullptr;
    int rc = scratch_on_current_device(&z);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    // column blocks of at most 32 right-hand sides that also fit the scratch
    const int64_t kfit = kNoAllocScratchFloats / g->n;
    for (int64_t c0 = 0; c0 < k;) {
        int kb = 32;
        while (kb > k - c0 || kb > kfit) kb >>= 1;
        const int v = pick_v_na(kb, ld, c0, x, y);
        switch (kb * 8 + v) {
            case 1 * 8 + 1: launch_pair<1, 1>(g, x + c0, ld, z, y + c0, st); break;
            case 2 * 8 + 1: launch_pair<2, 1>(g, x + c0, ld, z, y + c0, st); break;
            case 2 * 8 + 2: launch_pair<2, 2>(g, x + c0, ld, z, y + c0, st); break;
            case 4 * 8 + 1: launch_pair<4, 1>(g, x + c0, ld, z, y + c0, st); break;
            case 4 * 8 + 4: launch_pair<4, 4>(g, x + c0, ld, z, y + c0, st); break;
            case 8 * 8 + 1: launch_pair<8, 1>(g, x + c0, ld, z, y + c0, st); break;
            case 8 * 8 + 4: launch_pair<8, 4>(g, x + c0, ld, z, y + c0, st); break;
            case 16 * 8 + 1: launch_pair<16, 1>(g, x + c0, ld, z, y + c0, st); break;
            case 16 * 8 + 4: launch_pair<16, 4>(g, x + c0, ld, z, y + c0, st); break;
            case 32 * 8 + 1: launch_pair<32, 1>(g, x + c0, ld, z, y + c0, st); break;
            case 32 * 8 + 4: launch_pair<32, 4>(g, x + c0, ld, z, y + c0, st); break;
            default: return fail(BVG_ERR_INVALID_ARG, "bvg_spmv_xA_noalloc: no kernel for kb=%d v=%d", kb, v);
        }
        c0 += kb;
    }
    BVG_CUDA_TRY(cudaGetLastError());
    return BVG_OK;
}

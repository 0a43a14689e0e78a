// Many graphs in one launch: y_i = x_i A_i for every graph i of a batch.
//
// Small graphs leave most of the GPU idle and pay a launch each; here the
// tiles of all graphs form one grid. The chain step of every graph runs in one
// kernel, the gather of every graph in a second one (which may start while the
// first drains, through programmatic dependent launch), and the pair is
// replayed from a CUDA graph. Each CTA finds its graph by binary search over
// the first-tile offsets in a device table, then runs the same per-tile code
// as the one-graph product (over the graph's event or point columns, as its
// launch configuration says for the column block), so a batch result is
// bit-identical to the one-graph result for the same column block and vector
// width.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "fused.cuh"

using namespace bvg;

namespace bvg {

struct BatchEntry {
    const uint32_t* desc;
    const uint32_t* colp;  // event columns, or point columns when `points`
    const uint32_t* tent;
    const uint32_t* titem_ptr;
    const uint32_t* titem;
    const uint32_t* carry_ptr;
    const uint32_t* carry;
    const float* x;
    float* y;
    float* z;
    int64_t n;
    int64_t chain_tile0;   // first chain tile of this graph in the grid
    int64_t gather_tile0;  // first gather tile of this graph in the grid
    int points;            // 1: the gather reads point columns (no carry lists)
    const uint8_t* long_chunk;  // point columns: 128-column chunks holding a long column
    int64_t fx_tile0;      // one-vector blocks of a graph on the fused kernel: its first tile there
    FxArgs fx;             // that graph's fused-kernel arguments (x, y set per column block)
};

// Largest i with tab[i].tile0 <= blk (graphs with no rows are not in the
// table; a graph with no tiles in this grid shares its tile0 with the next
// graph, which the search then picks). WHICH: 0 chain, 1 gather, 2 fused.
template <int WHICH>
__device__ __forceinline__ int find_graph(const BatchEntry* __restrict__ tab, int count, int64_t blk) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int64_t t0 = WHICH == 0 ? tab[mid].chain_tile0 : (WHICH == 1 ? tab[mid].gather_tile0 : tab[mid].fx_tile0);
        if (t0 <= blk) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// One-vector column block of the graphs that use the fused kernel: every
// such graph's tiles in one grid, each CTA the same tile code as the
// one-graph product (bit-identical results).
__global__ void __launch_bounds__(kFxNT, 6) k_fx_batch(const BatchEntry* __restrict__ tab, int count, int64_t ld,
                                                  int64_t c0) {
    __shared__ __align__(16) FxSmem S;
    const BatchEntry& e = tab[find_graph<2>(tab, count, blockIdx.x)];
    FxArgs fa = e.fx;
    fa.x = e.x + c0;
    fa.ldx = ld;
    fa.y = e.y + c0;
    fa.ldy = ld;
    PrArgs pa{};
    fx_tile<0>((int64_t)blockIdx.x - e.fx_tile0, fa, pa, S);
}

template <int KB, int V>
__global__ void __launch_bounds__(256) k_chain_batch(const BatchEntry* __restrict__ tab, int count, int64_t ld,
                                                     int64_t c0) {
    asm volatile("griddepcontrol.launch_dependents;");
    const BatchEntry e = tab[find_graph<0>(tab, count, blockIdx.x)];
    chain_tile<KB, V>((int64_t)blockIdx.x - e.chain_tile0, e.desc, e.x + c0, ld, nullptr, e.z, KB, e.n);
}

template <int KB, int V>
__global__ void __launch_bounds__(GatherShape<KB, V>::NT) k_gather_batch(const BatchEntry* __restrict__ tab, int count, int64_t ld,
                                                      int64_t c0) {
    const BatchEntry e = tab[find_graph<1>(tab, count, blockIdx.x)];
    PrArgs pa{};
    df unused = df_zero();
    const int64_t blk = (int64_t)blockIdx.x - e.gather_tile0;
    if (e.points)
        gather_tile<KB, V, 0, false>(blk, e.colp, e.tent, e.titem_ptr, e.titem, nullptr, nullptr, e.long_chunk, e.z, KB,
                                     e.y + c0, ld, e.n, pa, unused);
    else
        gather_tile<KB, V, 0, true>(blk, e.colp, e.tent, e.titem_ptr, e.titem, e.carry_ptr, e.carry, nullptr, e.z, KB,
                                    e.y + c0, ld, e.n, pa, unused);
}

}  // namespace bvg

struct bvg_batch {
    std::vector<const bvg_dev_graph*> graphs;  // the graphs with n > 0, in input order
    std::vector<int> slot;                     // input index of each of them
    int32_t count_in = 0;
    int64_t total_n = 0, total_m = 0;
    int device = 0;
    float* z = nullptr;  // pushed weights of every graph, total_n x zk
    int64_t zk = 0;
    static constexpr int kRing = 4;
    BatchEntry* table = nullptr;  // device table (one per column block), fixed address for the CUDA graph
    int table_blocks = 0;
    BatchEntry* host_ring = nullptr;  // pinned staging, kRing slots of table_blocks * count entries
    cudaEvent_t ring_ev[kRing] = {};
    int ring_next = 0;
    // CUDA graph of the launches, and the signature it was captured for
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;
    int key_k = 0;
    std::vector<int> key_vs;  // vector width of each column block
    const void* key_table = nullptr;
    cudaEvent_t done_ev = nullptr;  // recorded after each call (orders calls across streams)
    bool called = false;
};

namespace bvg {

static int batch_fail_cuda(cudaError_t e, const char* what) {
    cudaGetLastError();
    return fail(BVG_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define BVG_BATCH_TRY(expr, what)                               \
    do {                                                        \
        cudaError_t e_ = (expr);                                \
        if (e_ != cudaSuccess) return batch_fail_cuda(e_, what); \
    } while (0)

template <int KB, int V>
static void chain_grid_tiles(int64_t n, int64_t& t) { t = (n + ChainShape<KB, V>::TILE - 1) / ChainShape<KB, V>::TILE; }
template <int KB, int V>
static void gather_grid_tiles(int64_t n, int64_t& t) { t = (n + GatherShape<KB, V>::T - 1) / GatherShape<KB, V>::T; }

template <int KB, int V>
static void launch_batch_pair(const BatchEntry* tab, int count, int64_t chain_tiles, int64_t gather_tiles,
                              int64_t ld, int64_t c0, cudaStream_t st) {
    if (chain_tiles == 0) return;  // every graph of this block runs on the fused kernel
    k_chain_batch<KB, V><<<(unsigned)chain_tiles, ChainShape<KB, V>::NT, 0, st>>>(tab, count, ld, c0);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)gather_tiles);
    cfg.blockDim = dim3(GatherShape<KB, V>::NT);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_gather_batch<KB, V>, tab, count, ld, c0);
}

#define BVG_BATCH_KV(FN, ...)                           \
    switch (kb * 8 + v) {                               \
        case 1 * 8 + 1: FN<1, 1>(__VA_ARGS__); break;   \
        case 2 * 8 + 1: FN<2, 1>(__VA_ARGS__); break;   \
        case 2 * 8 + 2: FN<2, 2>(__VA_ARGS__); break;   \
        case 4 * 8 + 1: FN<4, 1>(__VA_ARGS__); break;   \
        case 4 * 8 + 4: FN<4, 4>(__VA_ARGS__); break;   \
        case 8 * 8 + 1: FN<8, 1>(__VA_ARGS__); break;   \
        case 8 * 8 + 4: FN<8, 4>(__VA_ARGS__); break;   \
        case 16 * 8 + 1: FN<16, 1>(__VA_ARGS__); break; \
        case 16 * 8 + 4: FN<16, 4>(__VA_ARGS__); break; \
        case 32 * 8 + 1: FN<32, 1>(__VA_ARGS__); break; \
        case 32 * 8 + 4: FN<32, 4>(__VA_ARGS__); break; \
        default: break;                                 \
    }

// Column blocks of k right-hand sides: powers of two up to 32.
static std::vector<int> col_blocks(int k) {
    std::vector<int> out;
    for (int c0 = 0; c0 < k;) {
        int kb = 32;
        while (kb > k - c0) kb >>= 1;
        out.push_back(kb);
        c0 += kb;
    }
    return out;
}

static int ensure_tables(bvg_batch* b, int nblocks) {
    if (b->table_blocks >= nblocks) return BVG_OK;
    const size_t cnt = b->graphs.size();
    if (b->called) BVG_BATCH_TRY(cudaEventSynchronize(b->done_ev), "bvg_batch_spmv_xA");
    for (int r = 0; r < bvg_batch::kRing; r++)
        if (b->ring_ev[r]) BVG_BATCH_TRY(cudaEventSynchronize(b->ring_ev[r]), "bvg_batch_spmv_xA");
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->table) cudaFree(b->table);
    if (b->host_ring) cudaFreeHost(b->host_ring);
    b->table = nullptr;
    b->host_ring = nullptr;
    b->table_blocks = 0;
    cudaError_t e = cudaMalloc(&b->table, cnt * nblocks * sizeof(BatchEntry));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(BVG_ERR_OOM, "bvg_batch: table allocation failed");
    }
    e = cudaMallocHost(&b->host_ring, bvg_batch::kRing * cnt * nblocks * sizeof(BatchEntry));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(BVG_ERR_OOM, "bvg_batch: pinned staging allocation failed");
    }
    b->table_blocks = nblocks;
    return BVG_OK;
}

}  // namespace bvg

// ==================================================================== C ABI
extern "C" int bvg_batch_create(const bvg_dev_graph* const* gs, int32_t count, void* stream, bvg_batch** out) {
    (void)stream;
    if (!out) return fail(BVG_ERR_INVALID_ARG, "bvg_batch_create: out is NULL");
    *out = nullptr;
    if (!gs || count < 1) return fail(BVG_ERR_INVALID_ARG, "bvg_batch_create: need count >= 1 graphs");
    bvg_batch* b = new (std::nothrow) bvg_batch();
    if (!b) return fail(BVG_ERR_OOM, "bvg_batch_create: host allocation failed");
    b->count_in = count;
    cudaGetDevice(&b->device);
    for (int i = 0; i < count; i++) {
        if (!gs[i]) {
            delete b;
            return fail(BVG_ERR_INVALID_ARG, "bvg_batch_create: graph %d is NULL", i);
        }
        b->total_n += gs[i]->n;
        b->total_m += gs[i]->m;
        if (gs[i]->n > 0) {
            b->graphs.push_back(gs[i]);
            b->slot.push_back(i);
        }
    }
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->done_ev, cudaEventDisableTiming)) != cudaSuccess) {
        bvg_free_batch(b);
        return batch_fail_cuda(e, "bvg_batch_create");
    }
    for (int r = 0; r < bvg_batch::kRing; r++) {
        if ((e = cudaEventCreateWithFlags(&b->ring_ev[r], cudaEventDisableTiming)) != cudaSuccess) {
            bvg_free_batch(b);
            return batch_fail_cuda(e, "bvg_batch_create");
        }
    }
    *out = b;
    return BVG_OK;
}

extern "C" int bvg_batch_size(const bvg_batch* b, int32_t* count, int64_t* total_n, int64_t* total_m) {
    if (!b) return fail(BVG_ERR_INVALID_ARG, "bvg_batch_size: NULL batch");
    if (count) *count = b->count_in;
    if (total_n) *total_n = b->total_n;
    if (total_m) *total_m = b->total_m;
    return BVG_OK;
}

extern "C" int bvg_batch_spmv_xA(bvg_batch* b, const float* const* xs, float* const* ys, int32_t k, void* stream) {
    if (!b || !xs || !ys) return fail(BVG_ERR_INVALID_ARG, "bvg_batch_spmv_xA: NULL argument");
    if (k < 1) return fail(BVG_ERR_INVALID_ARG, "bvg_batch_spmv_xA: k < 1");
    const int cnt = (int)b->graphs.size();
    if (cnt == 0) return BVG_OK;
    int dev = 0;
    BVG_BATCH_TRY(cudaGetDevice(&dev), "bvg_batch_spmv_xA");
    if (dev != b->device) return fail(BVG_ERR_INVALID_ARG, "bvg_batch_spmv_xA: batch was created on device %d", b->device);
    for (int i = 0; i < cnt; i++) {
        const float* x = xs[b->slot[i]];
        float* y = ys[b->slot[i]];
        if (!x || !y) return fail(BVG_ERR_INVALID_ARG, "bvg_batch_spmv_xA: graph %d has a NULL vector", b->slot[i]);
        if ((uintptr_t)x % 4 || (uintptr_t)y % 4) return fail(BVG_ERR_INVALID_ARG, "bvg_batch_spmv_xA: misaligned");
        if (x == y) return fail(BVG_ERR_INVALID_ARG, "bvg_batch_spmv_xA: x and y of graph %d alias", b->slot[i]);
    }
    const std::vector<int> blocks = col_blocks(k);
    const int nb = (int)blocks.size();
    // vector width of each column block: the widest one that every graph's
    // x and y allow (the same rule as the one-graph product)
    std::vector<int> vs(nb);
    {
        int64_t c0 = 0;
        for (int bi = 0; bi < nb; bi++) {
            const int kb = blocks[bi];
            auto ok = [&](int v) {
                if (kb % v || k % v || c0 % v) return false;
                for (int i = 0; i < cnt; i++)
                    if ((uintptr_t)(xs[b->slot[i]] + c0) % (4 * v) || (uintptr_t)(ys[b->slot[i]] + c0) % (4 * v))
                        return false;
                return true;
            };
            vs[bi] = (kb >= 4 && ok(4)) ? 4 : ((kb == 2 && ok(2)) ? 2 : 1);
            c0 += kb;
        }
    }
    int rc;
    if ((rc = ensure_tables(b, nb))) return rc;
    // point columns a graph's configuration asks for (built once, synchronous)
    for (int bi = 0; bi < nb; bi++)
        for (int i = 0; i < cnt; i++)
            if (want_points(b->graphs[i], blocks[bi]) &&
                (rc = ensure_points(const_cast<bvg_dev_graph*>(b->graphs[i]), stream)))
                return rc;
    const int zk = blocks[0];  // the widest column block
    if (b->zk < zk) {
        if (b->z) {
            if (b->called) BVG_BATCH_TRY(cudaEventSynchronize(b->done_ev), "bvg_batch_spmv_xA");
            cudaFree(b->z);
        }
        b->z = nullptr;
        b->zk = 0;
        cudaError_t e = cudaMalloc(&b->z, (size_t)b->total_n * zk * sizeof(float));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(BVG_ERR_OOM, "bvg_batch_spmv_xA: z allocation failed");
        }
        b->zk = zk;
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
    }
    // fill a pinned staging slot with the table of every column block
    const int r = b->ring_next;
    b->ring_next = (r + 1) % bvg_batch::kRing;
    BVG_BATCH_TRY(cudaEventSynchronize(b->ring_ev[r]), "bvg_batch_spmv_xA");
    BatchEntry* h = b->host_ring + (size_t)r * cnt * b->table_blocks;
    std::vector<int64_t> chain_tiles(nb), gather_tiles(nb), fx_tiles(nb);
    for (int bi = 0; bi < nb; bi++) {
        const int kb = blocks[bi], v = vs[bi];
        int64_t ct = 0, gt = 0, ft = 0, zoff = 0;
        for (int i = 0; i < cnt; i++) {
            const bvg_dev_graph* g = b->graphs[i];
            BatchEntry& e = h[(size_t)bi * cnt + i];
            e.fx_tile0 = ft;
            e.chain_tile0 = ct;
            e.gather_tile0 = gt;
            if (use_fused(g, kb)) {  // the same choice as the one-graph product
                e.fx = fused_args(g, nullptr, 1, nullptr, nullptr, 1);
                e.x = xs[b->slot[i]];
                e.y = ys[b->slot[i]];
                e.n = g->n;
                ft += (g->n + kFxT - 1) / kFxT;
                continue;
            }
            e.fx = FxArgs{};
            e.desc = g->desc;
            e.points = use_points(g, kb) ? 1 : 0;
            e.colp = e.points ? g->pcolp : g->colp;
            e.tent = e.points ? g->pcent : g->tent;
            e.titem_ptr = e.points ? g->ptitem_ptr : g->titem_ptr;
            e.titem = e.points ? g->ptitem : g->titem;
            e.long_chunk = e.points ? g->plong : nullptr;
            e.carry_ptr = g->carry_ptr;
            e.carry = g->carry;
            e.x = xs[b->slot[i]];
            e.y = ys[b->slot[i]];
            e.z = b->z + zoff;
            e.n = g->n;
            e.chain_tile0 = ct;
            e.gather_tile0 = gt;
            int64_t t1 = 0, t2 = 0;
            BVG_BATCH_KV(chain_grid_tiles, g->n, t1);
            BVG_BATCH_KV(gather_grid_tiles, g->n, t2);
            ct += t1;
            gt += t2;
            zoff += g->n * kb;
        }
        chain_tiles[bi] = ct;
        gather_tiles[bi] = gt;
        fx_tiles[bi] = ft;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // a call on another stream than the last one waits for it (the table is shared)
    if (b->called) BVG_BATCH_TRY(cudaStreamWaitEvent(st, b->done_ev, 0), "bvg_batch_spmv_xA");
    BVG_BATCH_TRY(cudaMemcpyAsync(b->table, h, (size_t)nb * cnt * sizeof(BatchEntry), cudaMemcpyHostToDevice, st),
                  "bvg_batch_spmv_xA");
    BVG_BATCH_TRY(cudaEventRecord(b->ring_ev[r], st), "bvg_batch_spmv_xA");
    // the launches of all column blocks, captured once per signature
    if (!b->exec || b->key_k != k || b->key_vs != vs || b->key_table != b->table) {
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        BVG_BATCH_TRY(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal), "bvg_batch capture");
        int64_t c0 = 0;
        for (int bi = 0; bi < nb; bi++) {
            const int kb = blocks[bi], v = vs[bi];
            if (fx_tiles[bi] > 0)
                k_fx_batch<<<(unsigned)fx_tiles[bi], kFxNT, 0, b->cap_stream>>>(b->table + (size_t)bi * cnt, cnt,
                                                                               (int64_t)k, c0);
            BVG_BATCH_KV(launch_batch_pair, b->table + (size_t)bi * cnt, cnt, chain_tiles[bi], gather_tiles[bi],
                         (int64_t)k, c0, b->cap_stream);
            c0 += kb;
        }
        cudaError_t le = cudaGetLastError();
        cudaError_t ce = cudaStreamEndCapture(b->cap_stream, &graph);
        if (le != cudaSuccess || ce != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return batch_fail_cuda(le != cudaSuccess ? le : ce, "bvg_batch capture");
        }
        cudaError_t ie = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            b->exec = nullptr;
            return batch_fail_cuda(ie, "bvg_batch instantiate");
        }
        b->key_k = k;
        b->key_vs = vs;
        b->key_table = b->table;
    }
    BVG_BATCH_TRY(cudaGraphLaunch(b->exec, st), "bvg_batch_spmv_xA");
    BVG_BATCH_TRY(cudaEventRecord(b->done_ev, st), "bvg_batch_spmv_xA");
    b->called = true;
    return BVG_OK;
}

extern "C" void bvg_free_batch(bvg_batch* b) {
    if (!b) return;
    if (b->called) cudaEventSynchronize(b->done_ev);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (cudaEvent_t e : b->ring_ev)
        if (e) cudaEventDestroy(e);
    if (b->done_ev) cudaEventDestroy(b->done_ev);
    if (b->table) cudaFree(b->table);
    if (b->host_ring) cudaFreeHost(b->host_ring);
    if (b->z) cudaFree(b->z);
    delete b;
}

// C-ABI entry points of the device side: upload of the BV-delta layout,
// products, PageRank driver.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "fused.cuh"
#include "pull_fused.cuh"

using namespace bvg;

namespace bvg {

// ----------------------------------------------------------------- helpers
static int dev_alloc(void** p, size_t bytes, int64_t* total) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (inject_alloc_failure()) return fail(BVG_ERR_OOM, "cudaMalloc(%zu): injected failure", bytes);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? BVG_ERR_OOM : BVG_ERR_CUDA, "cudaMalloc(%zu): %s", bytes,
                    cudaGetErrorString(e));
    }
    if (total) *total += (int64_t)bytes;
    return BVG_OK;
}

template <class T>
static int upload_vec(T** dst, const std::vector<T>& v, cudaStream_t st, int64_t* total) {
    int rc = dev_alloc((void**)dst, v.size() * sizeof(T), total);
    if (rc) return rc;
    if (!v.empty()) BVG_CUDA_TRY(cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    return BVG_OK;
}

static int device_of(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return -2;
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return -1;
    return at.device;
}

// Largest power of two <= min(32, r).
static int block_k(int64_t r) {
    int kb = 32;
    while (kb > r) kb >>= 1;
    return kb;
}

// Vector width usable for a column block starting at `col` of buffers with
// leading dimension ld.
static int pick_v(int kb, int64_t ld, int64_t col, std::initializer_list<const void*> ptrs) {
    auto ok = [&](int v) {
        if (kb % v || ld % v || col % v) return false;
        for (const void* p : ptrs)
            if (p && ((uintptr_t)((const float*)p + col) % (4 * v))) return false;
        return true;
    };
    if (kb >= 4 && ok(4)) return 4;
    if (kb == 2 && ok(2)) return 2;
    return 1;
}

#define BVG_KV_CASES(FN, ...)                              \
    switch (kb * 8 + v) {                                  \
        case 1 * 8 + 1: FN<1, 1>(__VA_ARGS__); break;      \
        case 2 * 8 + 1: FN<2, 1>(__VA_ARGS__); break;      \
        case 2 * 8 + 2: FN<2, 2>(__VA_ARGS__); break;      \
        case 4 * 8 + 1: FN<4, 1>(__VA_ARGS__); break;      \
        case 4 * 8 + 4: FN<4, 4>(__VA_ARGS__); break;      \
        case 8 * 8 + 1: FN<8, 1>(__VA_ARGS__); break;      \
        case 8 * 8 + 4: FN<8, 4>(__VA_ARGS__); break;      \
        case 16 * 8 + 1: FN<16, 1>(__VA_ARGS__); break;    \
        case 16 * 8 + 4: FN<16, 4>(__VA_ARGS__); break;    \
        case 32 * 8 + 1: FN<32, 1>(__VA_ARGS__); break;    \
        case 32 * 8 + 4: FN<32, 4>(__VA_ARGS__); break;    \
        default: break;                                    \
    }

constexpr int kThreads = 256;

// Rows per CTA: the halo of kHalo rows is recomputed by two CTAs, so tiles
// stay large; shared memory grows with kb, and the tile is halved until the
// row sums (tile + kHalo rows x kb floats) fit in 200 KB.
static int pull_tile(int kb, const LaunchCfg& c) {
    int t = kb <= 4 ? c.pull_tile : std::max(128, c.pull_tile / 2);
    while (t > 64 && (size_t)(t + kHalo) * kb * sizeof(float) > 200 * 1024) t /= 2;
    return t;
}
// Columns per CTA of the gather kernel (k_gather's GatherShape).
static int gather_tile(int kb, int v, const LaunchCfg&) {
    const int G = kb / v, NT = G >= 8 ? 512 : 256, NG = NT / G, CPT = std::max(2, 128 / NG);
    return NG * CPT;
}

// Launch with programmatic stream serialization: the kernel may start while
// the previous kernel on the stream finishes; it waits (griddepcontrol.wait)
// before reading that kernel's output.
template <class... KArgs, class... Args>
static void launch_pdl(int pdl, void (*kernel)(KArgs...), int64_t grid, int block, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <class K>
static void set_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return;
    static std::mutex mu;
    static std::vector<std::pair<const void*, size_t>> done;
    std::lock_guard<std::mutex> lk(mu);
    for (auto& d : done)
        if (d.first == (const void*)kernel && d.second >= bytes) return;
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    done.push_back({(const void*)kernel, bytes});
}

// ----------------------------------------------------------------- tracing
struct Tracer {
    static constexpr int kPool = 65536;
    std::vector<cudaEvent_t> ev;  // 2 * kPool
    struct Rec {
        const char* name;
        int slot;
    };
    std::vector<Rec> recs;
    int next = 0;
    bool on = false;
};

struct TraceScope {
    Tracer* t;
    int slot = -1;
    cudaStream_t st;
    TraceScope(const bvg_dev_graph* g, const char* name, cudaStream_t s) : t(g->tracer), st(s) {
        if (t && t->on && t->next < Tracer::kPool) {
            slot = t->next++;
            t->recs.push_back({name, slot});
            cudaEventRecord(t->ev[2 * slot], st);
        }
    }
    ~TraceScope() {
        if (slot >= 0) cudaEventRecord(t->ev[2 * slot + 1], st);
    }
};

// ----------------------------------------------------------------- launchers
template <int KB, int V>
static void launch_pull(const bvg_dev_graph* g, const float* x, int64_t ldx, float* y, int64_t ldy, bool prefix,
                        cudaStream_t st) {
    PrefixArgs pf{};
    if (prefix) {
        using Sh = PrefixShape<KB, V>;
        const int64_t nb = (g->n + 1 + Sh::PB - 1) / Sh::PB;
        float* lhi = g->s.pre[0];
        float* llo = g->s.pre[1];
        float* bhi = g->s.pre[2];
        float* blo = g->s.pre[3];
        {
            TraceScope ts(g, "prefix_local", st);
            k_prefix_local<KB, V><<<(unsigned)nb, 256, 0, st>>>(x, ldx, lhi, llo, bhi, blo, g->n);
        }
        {
            TraceScope ts(g, "prefix_blocks", st);
            k_prefix_blocks<KB><<<1, 256, 0, st>>>(bhi, blo, (int)nb);
        }
        pf = PrefixArgs{lhi, llo, bhi, blo, Sh::PB, 0};
    }
    float* part = g->part;
    if (g->nitems > 0) {
        constexpr int G = KB / V;
        const int64_t grid = (g->nitems + 256 / G - 1) / (256 / G);
        TraceScope ts(g, "pull_items", st);
        switch (g->pull_built_item) {
            case 4: k_pull_items<KB, V, 4><<<(unsigned)grid, 256, 0, st>>>(g->pent, g->istart, g->nitems, x, ldx, part); break;
            case 16: k_pull_items<KB, V, 16><<<(unsigned)grid, 256, 0, st>>>(g->pent, g->istart, g->nitems, x, ldx, part); break;
            default: k_pull_items<KB, V, 8><<<(unsigned)grid, 256, 0, st>>>(g->pent, g->istart, g->nitems, x, ldx, part); break;
        }
    }
    const int tile = pull_tile(KB, g->cfg);
    const size_t smem = (size_t)(tile + kHalo) * KB * sizeof(float);
    set_smem(k_pull_rows<KB, V>, smem);
    const int64_t grid = (g->n + tile - 1) / tile;
    TraceScope ts(g, "pull_rows", st);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = g->nitems > 0 ? 1 : 0;
    cudaLaunchKernelEx(&cfg, k_pull_rows<KB, V>, (const uint8_t*)g->meta, (const uint32_t*)g->irow, (const float*)part,
                       (const uint32_t*)g->lrow, (const uint32_t*)g->lint, x, ldx, y, ldy, g->n, tile, pf);
}

template <int KB, int V>
static void launch_chain(const bvg_dev_graph* g, const float* x, int64_t ldx, const float* rowscale, float* z,
                         int64_t ldz, const PrState* pst, cudaStream_t st) {
    const int64_t grid = (g->n + ChainShape<KB, V>::TILE - 1) / ChainShape<KB, V>::TILE;
    TraceScope ts(g, pst ? "pr_chain" : "push_chain", st);
    k_chain<KB, V><<<(unsigned)grid, ChainShape<KB, V>::NT, 0, st>>>(g->desc, x, ldx, rowscale, z, ldz, g->n, pst);
}

// Whether the gather of a kb-wide column block reads the point columns
// (which ensure_points has built when this is true).
bool use_points(const bvg_dev_graph* g, int kb) {
    (void)kb;
    if (g->pcol_state != 1) return false;
    return g->cfg.push_points != 0;
}
bool want_points(const bvg_dev_graph* g, int kb) {
    (void)kb;
    if (g->pcol_state < 0) return false;
    return g->cfg.push_points != 0;
}

// Whether a one-vector column block runs as the fused kernel (fused.cuh): by
// default when no column tile reads rows outside its window (graphs with
// locality). The kernel runs as one wave, so a single tile on the slow
// far-row path sets its time; then the two-kernel product serves. It needs
// the point columns for its compensated path.
bool use_fused(const bvg_dev_graph* g, int kb) {
    if (kb != 1 || g->pcol_state != 1 || !g->tile_win) return false;
    if (g->cfg.push_fused == 0) return false;
    return g->cfg.push_fused == 1 || g->fx_far_tiles == 0;
}

FxArgs fused_args(const bvg_dev_graph* g, const float* x, int64_t ldx, const float* rowscale, float* y,
                   int64_t ldy) {
    FxArgs fa{};
    fa.desc = g->desc;
    fa.colp = g->colp;
    fa.tent16 = g->tent16;
    fa.carry_ptr = g->carry_ptr;
    fa.carry = g->carry;
    fa.pcolp = g->pcolp;
    fa.pcent = g->pcent;
    fa.tile_win = (const uint4*)g->tile_win;
    fa.lane_cols = g->lane_cols;
    fa.row_order = g->row_order;
    fa.row_groups = g->row_groups;
    fa.x = x;
    fa.ldx = ldx;
    fa.rowscale = rowscale;
    fa.y = y;
    fa.ldy = ldy;
    fa.n = g->n;
    fa.err = g->err;
    fa.tile0 = 0;
    return fa;
}

// Whether the one-vector pull runs as one kernel (pull_fused.cuh): its tables
// were built (every row tile's x window and work items fit the kernel).
bool use_pull_fused(const bvg_dev_graph* g, int kb) {
    return kb == 1 && g->cfg.pull_fused != 0 && g->px_ok;
}

PxArgs pull_fused_args(const bvg_dev_graph* g, const float* x, int64_t ldx, float* y, int64_t ldy) {
    PxArgs pa{};
    pa.irow = g->px_irow;
    pa.istart = g->px_istart;
    pa.pent = g->px_pent;
    pa.ptile = (const uint2*)g->px_tile;
    pa.meta = g->meta;
    pa.x = x;
    pa.ldx = ldx;
    pa.y = y;
    pa.ldy = ldy;
    pa.n = g->n;
    return pa;
}

static void launch_fused(const bvg_dev_graph* g, const float* x, int64_t ldx, float* y, int64_t ldy,
                         cudaStream_t st, int64_t tile0 = 0, int64_t tile1 = -1) {
    if (tile1 < 0) tile1 = (g->n + kFxT - 1) / kFxT;
    PrArgs pa{};
    TraceScope ts(g, "push_fused", st);
    FxArgs fa = fused_args(g, x, ldx, nullptr, y, ldy);
    fa.tile0 = tile0;
    k_push_fx<0><<<(unsigned)(tile1 - tile0), kFxNT, 0, st>>>(fa, pa);
}

// x A (one right-hand side) for the columns [col0, col1) only, when the
// fused kernel serves this graph and the range is made of whole column
// tiles (col0 a multiple of kFxT, col1 one too or n): the other columns of y
// are not written. Returns BVG_ERR_UNSUPPORTED otherwise (nothing launched).
int spmv_xA_columns(const bvg_dev_graph* g, const float* x, float* y, int64_t col0, int64_t col1, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (!use_fused(g, 1) || col0 < 0 || col1 > g->n || col0 > col1 || col0 % kFxT ||
        (col1 % kFxT && col1 != g->n))
        return BVG_ERR_UNSUPPORTED;
    if (col0 < col1) launch_fused(g, x, 1, y, 1, st, col0 / kFxT, (col1 + kFxT - 1) / kFxT);
    BVG_CUDA_TRY(cudaGetLastError());
    return BVG_OK;
}

template <int KB, int V>
static void launch_gather(const bvg_dev_graph* g, const float* z, int64_t ldz, float* y, int64_t ldy, cudaStream_t st) {
    const int tile = gather_tile(KB, V, g->cfg);
    const int64_t grid = (g->n + tile - 1) / tile;
    PrArgs pa{};
    if (use_points(g, KB)) {
        TraceScope ts(g, "push_gather_pt", st);
        launch_pdl(g->cfg.gather_pdl, k_gather_pt<KB, V, 0>, grid, GatherShape<KB, V>::NT, st,
                   (const uint32_t*)g->pcolp, (const uint32_t*)g->pcent, (const uint32_t*)g->ptitem_ptr,
                   (const uint32_t*)g->ptitem, (const uint8_t*)g->plong, z, ldz, y, ldy, g->n, pa);
        return;
    }
    TraceScope ts(g, "push_gather", st);
    launch_pdl(g->cfg.gather_pdl, k_gather<KB, V, 0>, grid, GatherShape<KB, V>::NT, st, (const uint32_t*)g->colp,
               (const uint32_t*)g->tent, (const uint32_t*)g->titem_ptr, (const uint32_t*)g->titem,
               (const uint32_t*)g->carry_ptr, (const uint32_t*)g->carry, z, ldz, y, ldy,
               g->n, pa);
}
// CTAs of `kernel` (nt threads, static shared memory only) resident on the
// current device at once.
static int64_t resident_ctas(const void* kernel, int nt) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, nt, 0) != cudaSuccess) {
        cudaGetLastError();
        return INT64_MAX;  // one tile per CTA, as without the loop
    }
    return (int64_t)sms * std::max(per_sm, 1);
}

template <int KB, int V>
static void launch_gather_pr(const bvg_dev_graph* g, const float* z, int64_t ldz, const PrArgs& pa, cudaStream_t st) {
    const int tile = gather_tile(KB, V, g->cfg);
    const int64_t tiles = (g->n + tile - 1) / tile;
    // a resident grid: the CTAs loop over the tiles and reduce once each
    const bool pt = use_points(g, KB);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(tiles, resident_ctas(pt ? (const void*)k_gather_pt<KB, V, 1>
                                                                                   : (const void*)k_gather<KB, V, 1>,
                                                                                GatherShape<KB, V>::NT)));
    if (pt) {
        TraceScope ts(g, "pr_gather_pt", st);
        launch_pdl(g->cfg.gather_pdl, k_gather_pt<KB, V, 1>, grid, GatherShape<KB, V>::NT, st,
                   (const uint32_t*)g->pcolp, (const uint32_t*)g->pcent, (const uint32_t*)g->ptitem_ptr,
                   (const uint32_t*)g->ptitem, (const uint8_t*)g->plong, z, ldz, (float*)nullptr, (int64_t)0, g->n,
                   pa);
        return;
    }
    TraceScope ts(g, "pr_gather", st);
    launch_pdl(g->cfg.gather_pdl, k_gather<KB, V, 1>, grid, GatherShape<KB, V>::NT, st, (const uint32_t*)g->colp,
               (const uint32_t*)g->tent, (const uint32_t*)g->titem_ptr, (const uint32_t*)g->titem,
               (const uint32_t*)g->carry_ptr, (const uint32_t*)g->carry, z, ldz,
               (float*)nullptr, (int64_t)0, g->n, pa);
}
template <int KB, int V>
static void launch_pr_init(const bvg_dev_graph* g, const float* p_init, int64_t ldi, const PrArgs& pa,
                           cudaStream_t st) {
    // wide column blocks: 8 gather tiles per CTA (a CTA of one 128-column
    // tile spends more on its share of the reduction than on its columns)
    const int tile = gather_tile(KB, V, g->cfg) * (KB >= 8 ? 8 : 1);
    const int64_t grid = (g->n + tile - 1) / tile;
    TraceScope ts(g, "pr_init", st);
    k_pr_init<KB, V><<<(unsigned)grid, kThreads, 0, st>>>(p_init, ldi, g->n, tile, pa);
}

template <int KB, int V>
static void launch_pr_final(const bvg_dev_graph* g, const PrState* pst, float* out, cudaStream_t st) {
    const int G = KB / V;
    const int64_t rows_per_block = kThreads / G;
    int64_t grid = (g->n + rows_per_block - 1) / rows_per_block;
    if (grid > 4096) grid = 4096;
    TraceScope ts(g, "pr_final", st);
    k_pr_final<KB, V><<<(unsigned)grid, kThreads, 0, st>>>(g->s.q[0], g->s.q[1], KB, g->s.sc[0], g->s.sc[1], pst,
                                                            out, KB, g->n);
}

// Grows the z scratch to n x kb floats.
static void drop_pr_graph(bvg_dev_graph* g);

static int ensure_z(bvg_dev_graph* g, int kb) {
    if (g->s.kcap >= kb) return BVG_OK;
    drop_pr_graph(g);  // the captured PageRank updates read the old z
    if (g->s.z) cudaFree(g->s.z);
    g->s.z = nullptr;
    g->s.kcap = 0;
    int rc = dev_alloc((void**)&g->s.z, (size_t)g->n * kb * sizeof(float), nullptr);
    if (rc) return rc;
    g->s.kcap = kb;
    return BVG_OK;
}

// Prefix scratch for kb columns: L hi/lo ((n+1) x kb) and block starts.
static int ensure_prefix(bvg_dev_graph* g, int kb) {
    if (g->s.pre_kcap >= kb) return BVG_OK;
    for (float*& b : g->s.pre) {
        if (b) cudaFree(b);
        b = nullptr;
    }
    g->s.pre_kcap = 0;
    const int64_t nb = (g->n + 1 + 7) / 8 + 1;  // enough blocks for the smallest block (8 rows x 1 group)
    const size_t lbytes = (size_t)(g->n + 1) * kb * sizeof(float), bbytes = (size_t)nb * kb * sizeof(float);
    int rc;
    if ((rc = dev_alloc((void**)&g->s.pre[0], lbytes, nullptr)) || (rc = dev_alloc((void**)&g->s.pre[1], lbytes, nullptr)) ||
        (rc = dev_alloc((void**)&g->s.pre[2], bbytes, nullptr)) || (rc = dev_alloc((void**)&g->s.pre[3], bbytes, nullptr)))
        return rc;
    g->s.pre_kcap = kb;
    return BVG_OK;
}

static bool use_prefix(const bvg_dev_graph* g) {
    return g->nlint > 0 && g->cfg.pull_prefix != 0;  // only kept (long) intervals read the prefix
}

// Partial sums of the pull items for kb columns.
static int ensure_part(bvg_dev_graph* g, int kb) {
    if (g->part_kcap >= kb) return BVG_OK;
    if (g->part) cudaFree(g->part);
    g->part = nullptr;
    g->part_kcap = 0;
    int rc = dev_alloc((void**)&g->part, (size_t)std::max<int64_t>(g->nitems, 1) * kb * sizeof(float), nullptr);
    if (rc) return rc;
    g->part_kcap = kb;
    return BVG_OK;
}

// Builds the pull work items (see build_pull_items) from the host copy of the
// difference rows and copies them to the device, replacing earlier arrays;
// synchronous.
static int build_pull_items(bvg_dev_graph* g, int item, int min_len, int prefix_mode, cudaStream_t st) {
    PullItems P;
    int rc0 = build_pull_items(g->host_rowp.data(), g->host_ent.data(), g->n, item, min_len, P, prefix_mode < 0);
    if (rc0) return rc0;
    std::vector<uint32_t>& pent = P.pent;
    std::vector<uint32_t>& istart = P.istart;
    std::vector<uint32_t>& irow = P.irow;
    std::vector<uint32_t>& lrow = P.lrow;
    std::vector<uint32_t>& lint = P.lint;
    BVG_CUDA_TRY(cudaStreamSynchronize(st));  // earlier products may still read the old arrays
    for (uint32_t** b : {&g->pent, &g->istart, &g->irow, &g->lrow, &g->lint}) {
        if (*b) cudaFree(*b);
        *b = nullptr;
    }
    if (g->part) cudaFree(g->part);
    g->part = nullptr;
    g->part_kcap = 0;
    g->npent = (int64_t)pent.size();
    g->nitems = (int64_t)istart.size() - 1;
    g->nlint = (int64_t)lint.size() / 2;
    int rc;
    int64_t bytes = 0;
    if ((rc = upload_vec(&g->pent, pent, st, &bytes)) || (rc = upload_vec(&g->istart, istart, st, &bytes)) ||
        (rc = upload_vec(&g->irow, irow, st, &bytes)) || (rc = upload_vec(&g->lrow, lrow, st, &bytes)) ||
        (rc = upload_vec(&g->lint, lint, st, &bytes)) || (rc = ensure_part(g, 1)))
        return rc;
    BVG_CUDA_TRY(cudaStreamSynchronize(st));  // the host vectors go out of scope
    g->pull_bytes = bytes;
    g->pull_built_item = item;
    g->pull_built_minlen = min_len;
    g->pull_built_auto = prefix_mode < 0 ? 1 : 0;
    return BVG_OK;
}

// Builds the point columns (see build_point_cols) from the host copy of the
// difference rows and copies them to the device, once; synchronous. If they
// cannot be built (2^30 entries or more) the event columns serve from then on.
int ensure_points(bvg_dev_graph* g, void* stream) {
    if (g->pcol_state != 0) return BVG_OK;
    cudaStream_t st = (cudaStream_t)stream;
    PointCols P;
    int rc = build_point_cols(g->host_rowp.data(), g->host_ent.data(), g->n, P);
    if (rc == BVG_ERR_UNSUPPORTED) {
        g->pcol_state = -1;
        return BVG_OK;
    }
    if (rc) return rc;
    int64_t bytes = 0;
    if ((rc = upload_vec(&g->pcolp, P.colp, st, &bytes)) || (rc = upload_vec(&g->pcent, P.ent, st, &bytes)) ||
        (rc = upload_vec(&g->ptitem_ptr, P.titem_ptr, st, &bytes)) || (rc = upload_vec(&g->ptitem, P.titem, st, &bytes)) ||
        (rc = upload_vec(&g->plong, P.long_chunk, st, &bytes)))
        return rc;
    BVG_CUDA_TRY(cudaStreamSynchronize(st));  // the host vectors go out of scope
    g->npcent = (int64_t)P.ent.size();
    g->nptitem = (int64_t)P.titem.size();
    g->pcol_bytes = bytes;
    g->pcol_state = 1;
    return BVG_OK;
}

static int64_t max_grid(const bvg_dev_graph* g) {
    // largest grid of any launch that writes per-CTA partials
    int64_t best = 0;
    for (int kb = 1; kb <= 32; kb *= 2)
        for (int v : {1, 2, 4}) {
            if (v > kb || kb % v) continue;
            int t = gather_tile(kb, v, g->cfg);
            best = std::max(best, (g->n + t - 1) / t);
        }
    return std::max<int64_t>(best, 1);
}

static void drop_pr_graph(bvg_dev_graph* g) {
    if (g->s.pr_exec) cudaGraphExecDestroy((cudaGraphExec_t)g->s.pr_exec);
    g->s.pr_exec = nullptr;
}

static int ensure_pr(bvg_dev_graph* g, int kb) {
    int rc = ensure_z(g, kb);
    if (rc) return rc;
    if (g->s.pr_kcap < kb) {
        drop_pr_graph(g);
        for (float** b : {&g->s.q[0], &g->s.q[1], &g->s.p0}) {
            if (*b) cudaFree(*b);
            *b = nullptr;
        }
        g->s.pr_kcap = 0;
        for (float** b : {&g->s.q[0], &g->s.q[1], &g->s.p0}) {
            rc = dev_alloc((void**)b, (size_t)g->n * kb * sizeof(float), nullptr);
            if (rc) return rc;
        }
        g->s.pr_kcap = kb;
    }
    if (!g->s.st) {
        rc = dev_alloc((void**)&g->s.st, sizeof(PrState), nullptr);
        if (rc) return rc;
        rc = dev_alloc((void**)&g->s.seed, 32 * sizeof(int64_t), nullptr);
        if (rc) return rc;
        for (int p = 0; p < 2; p++) {
            rc = dev_alloc((void**)&g->s.sc[p], sc_bytes(), nullptr);
            if (rc) return rc;
        }
        int64_t cap = max_grid(g) * 3 * 32;
        rc = dev_alloc((void**)&g->s.partial, (size_t)cap * sizeof(double), nullptr);
        if (rc) return rc;
        rc = dev_alloc((void**)&g->s.gpartial, (size_t)(max_grid(g) / kPrGroup + 1) * 3 * 32 * sizeof(double), nullptr);
        if (rc) return rc;
        g->s.partial_cap = cap;
        BVG_CUDA_TRY(cudaMallocHost((void**)&g->s.host_state, sizeof(PrState) + 64 * sizeof(double)));
    }
    return BVG_OK;
}

// The pull product y = M x^T on a device graph whose pull arrays (meta,
// irow, istart, pent, lrow, lint, part) may live anywhere the caller put them
// (the streamed row blocks): column blocks of at most 32, no interval kept
// whole (no prefix of x). part must hold nitems x 32 floats.
int pull_view_product(const bvg_dev_graph* gv, const float* x, float* y, int32_t k, int64_t ld, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    for (int64_t c0 = 0; c0 < k;) {
        const int kb = block_k(k - c0);
        const int v = pick_v(kb, ld, c0, {x, y});
        BVG_KV_CASES(launch_pull, gv, x + c0, ld, y + c0, ld, false, st);
        c0 += kb;
    }
    BVG_CUDA_TRY(cudaGetLastError());
    return BVG_OK;
}

int check_vec(const bvg_dev_graph* g, const void* p, const char* what) {
    if (!p) return fail(BVG_ERR_INVALID_ARG, "%s is NULL", what);
    if ((uintptr_t)p % 4) return fail(BVG_ERR_INVALID_ARG, "%s is not 4-byte aligned", what);
    int d = device_of(p);
    if (d != g->device) return fail(BVG_ERR_INVALID_ARG, "%s is not device memory of device %d", what, g->device);
    return BVG_OK;
}

}  // namespace bvg

// =================================================================== upload
// FNV-1a over the layout's 32-bit words (and its sizes): equal layouts give
// equal keys in the autotune cache.
static uint64_t layout_fingerprint(const HostLayout& L, int64_t n, int64_t m) {
    uint64_t h = 0xcbf29ce484222325ULL;
    auto mix = [&](uint64_t w) {
        h ^= w;
        h *= 0x100000001b3ULL;
    };
    mix((uint64_t)n);
    mix((uint64_t)m);
    for (const std::vector<uint32_t>* v : {&L.desc, &L.rowp, &L.ent, &L.colp, &L.tent, &L.carry_ptr, &L.carry}) {
        mix(v->size());
        for (uint32_t w : *v) mix(w);
    }
    return h;
}

extern "C" int bvg_upload(const bvg_host_graph* hg, void* stream, bvg_dev_graph** out) {
    if (!hg || !out) return fail(BVG_ERR_INVALID_ARG, "bvg_upload: NULL argument");
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = hg->n;
    bvg_dev_graph* g = new (std::nothrow) bvg_dev_graph();
    if (!g) return fail(BVG_ERR_OOM, "bvg_upload: host allocation failed");
    int rc = BVG_OK;
    try {
        BVG_CUDA_TRY(cudaGetDevice(&g->device));
        const HostLayout* L = nullptr;
        if ((rc = get_layout(hg, &L))) {
            delete g;
            return rc;
        }
        g->n = n;
        g->m = hg->m;
        g->nwords = (int64_t)L->ent.size();
        g->mean_interval = hg->stats.intervals ? (double)hg->stats.interval_members / (double)hg->stats.intervals : 0.0;
        g->ntent = (int64_t)L->tent.size();
        g->ntitem = (int64_t)L->titem.size();
        g->ncarry = (int64_t)L->carry.size();
        g->fingerprint = layout_fingerprint(*L, n, hg->m);
        // descendant masks and column entries padded (8 and 4 words): the
        // fused kernel copies 16-byte aligned supersets of its ranges
        std::vector<uint32_t> desc_pad(L->desc), tent_pad(L->tent);
        desc_pad.resize(((size_t)n + 3) / 4 * 4 + 8, 0u);
        tent_pad.resize((L->tent.size() + 3) / 4 * 4 + 4, 0u);
        if ((rc = upload_vec(&g->meta, L->meta, st, &g->bytes)) || (rc = upload_vec(&g->desc, desc_pad, st, &g->bytes)) || (rc = upload_vec(&g->rowp, L->rowp, st, &g->bytes)) ||
            (rc = upload_vec(&g->ent, L->ent, st, &g->bytes)) || (rc = upload_vec(&g->colp, L->colp, st, &g->bytes)) ||
            (rc = upload_vec(&g->tent, tent_pad, st, &g->bytes)) ||
            (rc = upload_vec(&g->titem_ptr, L->titem_ptr, st, &g->bytes)) ||
            (rc = upload_vec(&g->titem, L->titem, st, &g->bytes)) ||
            (rc = upload_vec(&g->carry_ptr, L->carry_ptr, st, &g->bytes)) ||
            (rc = upload_vec(&g->carry, L->carry, st, &g->bytes)) ||
            (rc = upload_vec(&g->inv_outdeg, L->inv_outdeg, st, &g->bytes))) {
            bvg_free_dev(g);
            return rc;
        }
        g->host_rowp = L->rowp;
        g->host_ent = L->ent;
        if ((rc = build_pull_items(g, g->cfg.pull_item, g->cfg.prefix_min_len, g->cfg.pull_prefix, st))) {
            bvg_free_dev(g);
            return rc;
        }
        // the fused one-vector push: each tile's row window, the span of the
        // rows its entries and its open intervals come from (kFxW at most:
        // a tile reading a wider span is flagged and keeps a window around
        // its own columns)
        {
            const int64_t tiles = (n + kFxT - 1) / kFxT;
            std::vector<uint32_t> win((size_t)tiles * 4, 0u);
            // and the tile's entries as 16-bit window offsets (with the two
            // flags), for the tiles whose sources lie in their window
            std::vector<uint16_t> tent16((L->tent.size() + 7) / 8 * 8 + 8, (uint16_t)0);
            int64_t nfar = 0;
            for (int64_t t = 0; t < tiles; t++) {
                const int64_t a = t * kFxT, e = std::min<int64_t>(n, a + kFxT);
                int64_t lo = INT64_MAX, hi = -1;
                for (uint32_t q = L->colp[a]; q < L->colp[e]; q++) {
                    const int64_t k = L->tent[q] & kIdMask;
                    lo = std::min(lo, k);
                    hi = std::max(hi, k);
                }
                for (int64_t ct = a / kCarryTile; ct < (e + kCarryTile - 1) / kCarryTile; ct++)
                    for (uint32_t q = L->carry_ptr[ct]; q < L->carry_ptr[ct + 1]; q++) {
                        lo = std::min<int64_t>(lo, L->carry[q]);
                        hi = std::max<int64_t>(hi, L->carry[q]);
                    }
                uint32_t far = 0;
                if (hi < 0) {  // nothing to read
                    lo = a;
                    hi = a;
                } else if (hi + 1 - lo > kFxW) {
                    far = 1;
                    lo = std::max<int64_t>(0, std::min<int64_t>(a - (kFxW - kFxT) / 2, n - kFxW));
                    hi = std::min<int64_t>(n, lo + kFxW) - 1;
                }
                if (!far)
                    for (uint32_t q = L->colp[a]; q < L->colp[e]; q++)
                        tent16[q] = (uint16_t)(((L->tent[q] & kIdMask) - (uint32_t)lo) | ((L->tent[q] >> kIdBits) << 14));
                win[(size_t)t * 4] = (uint32_t)lo;
                win[(size_t)t * 4 + 1] = (uint32_t)(hi + 1);
                win[(size_t)t * 4 + 2] = far;
                nfar += far;
            }
            g->fx_tiles = tiles;
            g->fx_far_tiles = nfar;
            // each warp's columns (a group of kCarryTile) sorted by entry count,
            // most first, the q-th 32 in lane slot q: a warp's loop over slot q
            // runs as long as the longest column of that group, and the sum
            // of those maxima is the least an assignment of 4 columns per lane
            // gives
            const int64_t groups = (n + kCarryTile - 1) / kCarryTile;
            std::vector<uint32_t> lane_cols((size_t)groups * 32, 0u);
            std::vector<int> ord(kCarryTile);
            std::vector<uint32_t> cnt(kCarryTile);
            for (int64_t t = 0; t < groups; t++) {
                for (int o = 0; o < kCarryTile; o++) {
                    const int64_t j = t * kCarryTile + o;
                    cnt[o] = j < n ? L->colp[j + 1] - L->colp[j] : 0u;
                    ord[o] = o;
                }
                std::stable_sort(ord.begin(), ord.end(), [&](int u, int v) { return cnt[u] > cnt[v]; });
                for (int l = 0; l < 32; l++)
                    for (int q = 0; q < kCarryTile / 32; q++)
                        lane_cols[(size_t)t * 32 + l] |= (uint32_t)ord[q * 32 + l] << (8 * q);
            }
            // the chain weights' row order: each aligned block of kFxNT rows
            // sorted by descendant count, most first; the q-th 32 rows go to
            // warp (q + b) mod 8 of block b, so that the heaviest rows fall to
            // a different warp in each block
            const int64_t rblocks = (n + kFxNT - 1) / kFxNT;
            g->row_groups = (rblocks + 3) / 4;
            std::vector<uint32_t> row_order((size_t)g->row_groups * kFxNT, 0u);
            std::vector<int> rord(kFxNT), rcnt(kFxNT);
            for (int64_t b = 0; b < rblocks; b++) {
                for (int o = 0; o < kFxNT; o++) {
                    const int64_t r = b * kFxNT + o;
                    rcnt[o] = r < n ? __builtin_popcount(L->desc[r]) : -1;
                    rord[o] = o;
                }
                std::stable_sort(rord.begin(), rord.end(), [&](int u, int v) { return rcnt[u] > rcnt[v]; });
                for (int k = 0; k < kFxNT; k++) {
                    const int pos = (((k >> 5) + (int)(b & 7)) & 7) * 32 + (k & 31);
                    row_order[(size_t)(b >> 2) * kFxNT + pos] |= (uint32_t)rord[k] << (8 * (int)(b & 3));
                }
            }
            uint32_t* dwin = nullptr;
            if ((rc = upload_vec(&dwin, win, st, &g->bytes)) || (rc = upload_vec(&g->lane_cols, lane_cols, st, &g->bytes)) ||
                (rc = upload_vec(&g->row_order, row_order, st, &g->bytes)) ||
                (rc = upload_vec(&g->tent16, tent16, st, &g->bytes)) ||
                (rc = dev_alloc((void**)&g->err, sizeof(unsigned int), nullptr))) {
                if (dwin) cudaFree(dwin);
                bvg_free_dev(g);
                return rc;
            }
            g->tile_win = dwin;
            BVG_CUDA_TRY(cudaMemsetAsync(g->err, 0, sizeof(unsigned int), st));
        }
        // the one-vector pull (pull_fused.cuh): work items with every interval
        // expanded, each row tile's x window, and each entry as the offset of
        // its column in the window of the tile that owns its row
        {
            PullItems P;
            if ((rc = build_pull_items(L->rowp.data(), L->ent.data(), n, kPxItem, INT32_MAX, P, false))) {
                bvg_free_dev(g);
                return rc;
            }
            const int64_t ptiles = (n + kPxT - 1) / kPxT;
            std::vector<uint32_t> pwin((size_t)ptiles * 2, 0u);
            bool ok = P.lint.empty();
            for (int64_t t = 0; t < ptiles && ok; t++) {
                const int64_t a = t * kPxT, lo = std::max<int64_t>(0, a - kHalo), e = std::min<int64_t>(n, a + kPxT);
                const uint32_t k0 = P.irow[lo], k1 = P.irow[e];
                if (k1 - k0 > (uint32_t)kPxItemCap) ok = false;
                int64_t cmin = INT64_MAX, cmax = -1;
                for (uint32_t q = P.istart[k0]; q < P.istart[k1]; q++) {
                    const int64_t c = P.pent[q] & 0x7fffffffu;
                    cmin = std::min(cmin, c);
                    cmax = std::max(cmax, c);
                }
                if (cmax < 0) cmin = cmax = a;
                else cmax += 1;
                if (cmax - cmin > kPxW) ok = false;
                pwin[(size_t)t * 2] = (uint32_t)cmin;
                pwin[(size_t)t * 2 + 1] = (uint32_t)cmax;
            }
            std::vector<uint16_t> pd(ok ? P.pent.size() : 0);
            for (int64_t r = 0; r < n && ok; r++) {
                const int64_t w0 = pwin[(size_t)(r / kPxT) * 2];
                for (uint32_t q = P.istart[P.irow[r]]; q < P.istart[P.irow[r + 1]]; q++)
                    pd[q] = (uint16_t)(((P.pent[q] & 0x7fffffffu) - w0) | ((P.pent[q] >> 31) << 15));
            }
            if (ok) {
                uint32_t* dtile = nullptr;
                if ((rc = upload_vec(&g->px_irow, P.irow, st, &g->bytes)) ||
                    (rc = upload_vec(&g->px_istart, P.istart, st, &g->bytes)) ||
                    (rc = upload_vec(&g->px_pent, pd, st, &g->bytes)) || (rc = upload_vec(&dtile, pwin, st, &g->bytes))) {
                    if (dtile) cudaFree(dtile);
                    bvg_free_dev(g);
                    return rc;
                }
                g->px_tile = dtile;
                g->px_ok = 1;
                BVG_CUDA_TRY(cudaStreamSynchronize(st));  // the host vectors go out of scope
            }
        }
        // the point columns (the gather of every column block, and the fused
        // kernel's compensated path)
        if ((rc = ensure_points(g, st))) {
            bvg_free_dev(g);
            return rc;
        }
        // global + one per group of CTAs + the update gather's tile counter
        const size_t ncount = (size_t)(1 + max_grid(g) / kPrGroup + 1) + 1;
        if ((rc = ensure_z(g, 1)) || (rc = dev_alloc((void**)&g->s.counter, ncount * sizeof(unsigned int), nullptr))) {
            bvg_free_dev(g);
            return rc;
        }
        BVG_CUDA_TRY(cudaMemsetAsync(g->s.counter, 0, ncount * sizeof(unsigned int), st));
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            bvg_free_dev(g);
            return fail(BVG_ERR_CUDA, "bvg_upload: %s", cudaGetErrorString(e));
        }
    } catch (const std::bad_alloc&) {
        bvg_free_dev(g);
        return fail(BVG_ERR_OOM, "bvg_upload: host allocation failed");
    }
    *out = g;
    return BVG_OK;
}

extern "C" void bvg_free_dev(bvg_dev_graph* g) {
    if (!g) return;
    void* ptrs[] = {g->meta, g->desc, g->rowp, g->ent, g->colp, g->tent, g->titem_ptr, g->titem, g->carry_ptr, g->carry,
                    g->inv_outdeg, g->s.z,
                    g->s.q[0], g->s.q[1], g->s.sc[0], g->s.sc[1], g->s.st, g->s.seed, g->s.partial, g->s.counter, g->s.hx,
                    g->s.hy, g->s.p0, g->s.pre[0], g->s.pre[1], g->s.pre[2], g->s.pre[3],
                    g->s.feat_tmp, g->s.wfeat, g->s.gpartial, g->pent, g->istart, g->irow, g->lrow, g->lint, g->part,
                    g->pcolp, g->pcent, g->ptitem_ptr, g->ptitem, g->plong, g->tile_win, g->lane_cols, g->row_order, g->tent16, g->px_irow, g->px_istart,
                    g->px_pent, g->px_tile, g->err};
    drop_pr_graph(g);
    if (g->s.cap_stream) cudaStreamDestroy((cudaStream_t)g->s.cap_stream);
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (g->s.host_state) cudaFreeHost(g->s.host_state);
    if (g->tracer) {
        for (cudaEvent_t e : g->tracer->ev) cudaEventDestroy(e);
        delete g->tracer;
    }
    delete g;
}

extern "C" int bvg_trace_enable(bvg_dev_graph* g, int enable) {
    if (!g) return fail(BVG_ERR_INVALID_ARG, "bvg_trace_enable: NULL graph");
    if (enable && !g->tracer) {
        Tracer* t = new (std::nothrow) Tracer();
        if (!t) return fail(BVG_ERR_OOM, "bvg_trace_enable: host allocation failed");
        t->ev.resize(2 * Tracer::kPool);
        for (auto& e : t->ev) {
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                for (auto& f : t->ev)
                    if (f) cudaEventDestroy(f);
                delete t;
                return fail(BVG_ERR_CUDA, "bvg_trace_enable: cudaEventCreate failed");
            }
        }
        g->tracer = t;
    }
    if (g->tracer) g->tracer->on = enable != 0;
    return BVG_OK;
}

extern "C" int bvg_trace_read(bvg_dev_graph* g, bvg_trace_entry* out, int32_t cap, int32_t* count) {
    if (!g || !count || (cap > 0 && !out)) return fail(BVG_ERR_INVALID_ARG, "bvg_trace_read: bad argument");
    *count = 0;
    if (!g->tracer) return BVG_OK;
    Tracer* t = g->tracer;
    std::vector<bvg_trace_entry> agg;
    for (const auto& r : t->recs) {
        BVG_CUDA_TRY(cudaEventSynchronize(t->ev[2 * r.slot + 1]));
        float ms = 0.f;
        BVG_CUDA_TRY(cudaEventElapsedTime(&ms, t->ev[2 * r.slot], t->ev[2 * r.slot + 1]));
        auto it = std::find_if(agg.begin(), agg.end(), [&](const bvg_trace_entry& e) { return !strcmp(e.name, r.name); });
        if (it == agg.end()) {
            bvg_trace_entry e{};
            strncpy(e.name, r.name, sizeof(e.name) - 1);
            agg.push_back(e);
            it = agg.end() - 1;
        }
        it->launches++;
        it->total_ms += ms;
    }
    t->recs.clear();
    t->next = 0;
    for (int i = 0; i < (int)agg.size() && i < cap; i++) out[i] = agg[i];
    *count = (int32_t)std::min<size_t>(agg.size(), (size_t)std::max(cap, 0));
    return BVG_OK;
}

extern "C" int bvg_dev_size(const bvg_dev_graph* g, int64_t* n, int64_t* m) {
    if (!g) return fail(BVG_ERR_INVALID_ARG, "bvg_dev_size: NULL graph");
    if (n) *n = g->n;
    if (m) *m = g->m;
    return BVG_OK;
}

extern "C" int bvg_get_config(const bvg_dev_graph* g, bvg_launch_config* out) {
    if (!g || !out) return fail(BVG_ERR_INVALID_ARG, "bvg_get_config: NULL argument");
    out->pull_tile = g->cfg.pull_tile;
    out->pull_prefix = g->cfg.pull_prefix;
    out->prefix_min_len = g->cfg.prefix_min_len;
    out->gather_pdl = g->cfg.gather_pdl;
    out->col_block = g->cfg.col_block;
    out->pull_item = g->cfg.pull_item;
    out->push_points = g->cfg.push_points;
    out->push_fused = g->cfg.push_fused;
    out->pull_fused = g->cfg.pull_fused;
    return BVG_OK;
}

extern "C" int bvg_set_config(bvg_dev_graph* g, const bvg_launch_config* in) {
    if (!g || !in) return fail(BVG_ERR_INVALID_ARG, "bvg_set_config: NULL argument");
    if (in->pull_tile < 64 || in->pull_tile > kPullMaxTile || (in->pull_tile & (in->pull_tile - 1)) ||
        in->pull_prefix < -1 || in->pull_prefix > 1 || in->prefix_min_len < 1 || in->gather_pdl < 0 ||
        in->gather_pdl > 1 || in->col_block < 1 || in->col_block > 32 || (in->col_block & (in->col_block - 1)) ||
        (in->pull_item != 4 && in->pull_item != 8 && in->pull_item != 16) || in->push_points < -1 ||
        in->push_points > 1 || in->push_fused < -1 || in->push_fused > 1 || in->pull_fused < -1 ||
        in->pull_fused > 1)
        return fail(BVG_ERR_INVALID_ARG, "bvg_set_config: pull_tile a power of two in [64, 2048], pull_prefix in "
                                         "{-1,0,1}, prefix_min_len >= 1, gather_pdl in {0,1}, col_block a power "
                                         "of two in [1, 32], pull_item in {4, 8, 16}, push_points, push_fused "
                                         "and pull_fused in {-1,0,1}");
    if (in->pull_item != g->pull_built_item || in->prefix_min_len != g->pull_built_minlen ||
        (in->pull_prefix < 0 ? 1 : 0) != g->pull_built_auto) {
        int rc = build_pull_items(g, in->pull_item, in->prefix_min_len, in->pull_prefix, nullptr);
        if (rc) return rc;
    }
    if (in->gather_pdl != g->cfg.gather_pdl || in->push_points != g->cfg.push_points ||
        in->push_fused != g->cfg.push_fused)
        drop_pr_graph(g);  // the PageRank graph was captured with the old launch
    g->cfg.pull_tile = in->pull_tile;
    g->cfg.pull_prefix = in->pull_prefix;
    g->cfg.prefix_min_len = in->prefix_min_len;
    g->cfg.gather_pdl = in->gather_pdl;
    g->cfg.col_block = in->col_block;
    g->cfg.pull_item = in->pull_item;
    g->cfg.push_points = in->push_points;
    g->cfg.push_fused = in->push_fused;
    g->cfg.pull_fused = in->pull_fused;
    return BVG_OK;
}

extern "C" int bvg_dev_layout(const bvg_dev_graph* g, bvg_layout_info* out) {
    if (!g || !out) return fail(BVG_ERR_INVALID_ARG, "bvg_dev_layout: NULL argument");
    out->n = g->n;
    out->m = g->m;
    out->words = g->nwords;
    out->col_entries = g->ntent;
    out->carry_tiles = (g->n + kCarryTile - 1) / kCarryTile;
    out->carry_entries = g->ncarry;
    out->structure_bytes = g->bytes + g->pull_bytes + g->pcol_bytes;
    out->pull_entries = g->npent;
    out->pull_items = g->nitems;
    out->pull_intervals = g->nlint;
    out->tail_items = g->ntitem;
    out->point_entries = g->npcent;
    out->point_tail_items = g->nptitem;
    return BVG_OK;
}

// =================================================================== products
extern "C" int bvg_spmv_Ax(const bvg_dev_graph* g, const float* x, float* y, int32_t k, int64_t ld, void* stream) {
    if (!g) return fail(BVG_ERR_INVALID_ARG, "bvg_spmv_Ax: NULL graph");
    if (k < 1 || ld < k) return fail(BVG_ERR_INVALID_ARG, "bvg_spmv_Ax: need k >= 1 and ld >= k");
    if (g->n == 0) return BVG_OK;
    int rc;
    if ((rc = check_vec(g, x, "x")) || (rc = check_vec(g, y, "y"))) return rc;
    if (x == y) return fail(BVG_ERR_INVALID_ARG, "bvg_spmv_Ax: x and y must not alias");
    cudaStream_t st = (cudaStream_t)stream;
    bvg_dev_graph* gm = const_cast<bvg_dev_graph*>(g);
    if (k == 1 && use_pull_fused(g, 1)) {  // one vector: one launch
        TraceScope ts(g, "pull_fused", st);
        k_pull_fx<<<(unsigned)((g->n + kPxT - 1) / kPxT), kPxNT, 0, st>>>(pull_fused_args(g, x, ld, y, ld));
        BVG_CUDA_TRY(cudaGetLastError());
        return BVG_OK;
    }
    const bool prefix = use_prefix(g);
    for (int64_t c0 = 0; c0 < k; ) {
        const int kb = block_k(std::min<int64_t>(k - c0, g->cfg.col_block));
        if ((prefix && (rc = ensure_prefix(gm, kb))) || (rc = ensure_part(gm, kb))) return rc;
        const int v = pick_v(kb, ld, c0, {x, y});
        BVG_KV_CASES(launch_pull, g, x + c0, ld, y + c0, ld, prefix, st);
        c0 += kb;
    }
    BVG_CUDA_TRY(cudaGetLastError());
    return BVG_OK;
}

// x A on vectors the device can address (checked by the callers).
static int spmv_xA(bvg_dev_graph* g, const float* x, float* y, int32_t k, int64_t ld, void* stream) {
    int rc;
    cudaStream_t st = (cudaStream_t)stream;
    for (int64_t c0 = 0; c0 < k; ) {
        const int kb = block_k(std::min<int64_t>(k - c0, g->cfg.col_block));
        if (use_fused(g, kb)) {
            launch_fused(g, x + c0, ld, y + c0, ld, st);
            c0 += kb;
            continue;
        }
        if ((rc = ensure_z(g, kb))) return rc;
        if (want_points(g, kb) && (rc = ensure_points(g, st))) return rc;
        const int v = pick_v(kb, ld, c0, {x, y});
        BVG_KV_CASES(launch_chain, g, x + c0, ld, nullptr, g->s.z, kb, nullptr, st);
        BVG_KV_CASES(launch_gather, g, g->s.z, kb, y + c0, ld, st);
        c0 += kb;
    }
    BVG_CUDA_TRY(cudaGetLastError());
    return BVG_OK;
}

extern "C" int bvg_spmv_xA(const bvg_dev_graph* gc, const float* x, float* y, int32_t k, int64_t ld, void* stream) {
    bvg_dev_graph* g = const_cast<bvg_dev_graph*>(gc);
    if (!g) return fail(BVG_ERR_INVALID_ARG, "bvg_spmv_xA: NULL graph");
    if (k < 1 || ld < k) return fail(BVG_ERR_INVALID_ARG, "bvg_spmv_xA: need k >= 1 and ld >= k");
    if (g->n == 0) return BVG_OK;
    int rc;
    if ((rc = check_vec(g, x, "x")) || (rc = check_vec(g, y, "y"))) return rc;
    if (x == y) return fail(BVG_ERR_INVALID_ARG, "bvg_spmv_xA: x and y must not alias");
    return spmv_xA(g, x, y, k, ld, stream);
}

extern "C" int bvg_spmv_xA_host(const bvg_dev_graph* gc, const float* x_host, float* y_host, int32_t k,
                                void* stream) {
    bvg_dev_graph* g = const_cast<bvg_dev_graph*>(gc);
    if (!g || !x_host || !y_host) return fail(BVG_ERR_INVALID_ARG, "bvg_spmv_xA_host: NULL argument");
    if (k < 1) return fail(BVG_ERR_INVALID_ARG, "bvg_spmv_xA_host: k < 1");
    if (g->n == 0) return BVG_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (x_host == y_host) return fail(BVG_ERR_INVALID_ARG, "bvg_spmv_xA_host: x and y must not alias");
    // staged through device scratch: one copy each way. (Reading and writing
    // page-locked buffers in place through their device mapping instead was
    // no faster: the chain and gather kernels then ran 2.3x slower on the
    // CPU-GPU link than on HBM.)
    const int64_t need = g->n * (int64_t)k;
    if (g->s.stage_cap < need) {
        if (g->s.hx) cudaFree(g->s.hx);
        if (g->s.hy) cudaFree(g->s.hy);
        g->s.hx = g->s.hy = nullptr;
        g->s.stage_cap = 0;
        int rc;
        if ((rc = dev_alloc((void**)&g->s.hx, need * sizeof(float), nullptr)) ||
            (rc = dev_alloc((void**)&g->s.hy, need * sizeof(float), nullptr)))
            return rc;
        g->s.stage_cap = need;
    }
    BVG_CUDA_TRY(cudaMemcpyAsync(g->s.hx, x_host, need * sizeof(float), cudaMemcpyHostToDevice, st));
    int rc = spmv_xA(g, g->s.hx, g->s.hy, k, k, stream);
    if (rc) return rc;
    BVG_CUDA_TRY(cudaMemcpyAsync(y_host, g->s.hy, need * sizeof(float), cudaMemcpyDeviceToHost, st));
    BVG_CUDA_TRY(cudaStreamSynchronize(st));
    return BVG_OK;
}

extern "C" int bvg_device_check(const bvg_dev_graph* gc, void* stream) {
    bvg_dev_graph* g = const_cast<bvg_dev_graph*>(gc);
    if (!g) return fail(BVG_ERR_INVALID_ARG, "bvg_device_check: NULL graph");
    if (!g->err) return BVG_OK;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned int h = 0;
    BVG_CUDA_TRY(cudaMemcpyAsync(&h, g->err, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
    BVG_CUDA_TRY(cudaStreamSynchronize(st));
    if (h) {
        BVG_CUDA_TRY(cudaMemsetAsync(g->err, 0, sizeof(unsigned int), st));
        BVG_CUDA_TRY(cudaStreamSynchronize(st));
        return fail(BVG_ERR_TIMEOUT, "bvg_device_check: a bounded device wait ran out in an earlier launch");
    }
    return BVG_OK;
}

// =================================================================== PageRank
// The solve behind bvg_pagerank (dense teleport vectors p0, or uniform) and
// bvg_pagerank_seeds (one-hot teleport vectors given by their nodes, host
// array `seeds`; p0 is then NULL).
static int pagerank_run(const bvg_dev_graph* gc, const bvg_pr_params* params, const float* p0, const int64_t* seeds,
                        const float* p_init, int32_t k, float* p_out, int32_t* iters_out, double* resid_out,
                        void* stream) {
    bvg_dev_graph* g = const_cast<bvg_dev_graph*>(gc);
    if (!g || !p_out) return fail(BVG_ERR_INVALID_ARG, "bvg_pagerank: NULL graph or output");
    if (k != 1 && k != 2 && k != 4 && k != 8 && k != 16 && k != 32)
        return fail(BVG_ERR_UNSUPPORTED, "bvg_pagerank: k must be 1, 2, 4, 8, 16 or 32 (got %d)", k);
    if (!p0 && !seeds && k != 1)
        return fail(BVG_ERR_INVALID_ARG, "bvg_pagerank: uniform teleport (p0 = NULL) needs k = 1");
    if (seeds)
        for (int c = 0; c < k; c++)
            if (seeds[c] < 0 || seeds[c] >= g->n)
                return fail(BVG_ERR_INVALID_ARG, "bvg_pagerank_seeds: seed %d is %lld, outside [0, %lld)", c,
                            (long long)seeds[c], (long long)g->n);
    const double damping = params && params->damping > 0 ? params->damping : 0.85;
    const double tol = params ? params->tol_l1 : 1e-8;
    const int max_iter = params && params->max_iter > 0 ? params->max_iter : 1000;
    const int dangling = params ? params->dangling : 0;
    if (!(damping > 0 && damping < 1) || !(tol >= 0) || (dangling != 0 && dangling != 1))
        return fail(BVG_ERR_INVALID_ARG, "bvg_pagerank: need 0 < damping < 1, tol >= 0, dangling in {0,1}");
    if (g->n == 0) {
        if (iters_out) *iters_out = 0;
        return BVG_OK;
    }
    int rc;
    if ((rc = check_vec(g, p_out, "p_out"))) return rc;
    if (p0 && (rc = check_vec(g, p0, "p0"))) return rc;
    if (p_init && (rc = check_vec(g, p_init, "p_init"))) return rc;
    if ((rc = ensure_pr(g, k))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int kb = k;
    if (want_points(g, kb) && (rc = ensure_points(g, st))) return rc;
    const int v = pick_v(kb, kb, 0, {p0, p_init, p_out, g->s.q[0], g->s.q[1]});

    PrState hs{0, 0, 0, max_iter, tol};
    PrState* pst = (PrState*)g->s.st;
    BVG_CUDA_TRY(cudaMemcpyAsync(pst, &hs, sizeof(hs), cudaMemcpyHostToDevice, st));
    // the update graph reads the teleport vectors from the handle's own copy:
    // dense vectors copied; one-hot vectors as their k nodes (k >= 2), or
    // written out densely for one vector (the one-launch update reads p0)
    static const float kOne = 1.0f;
    const float* p0_dev = nullptr;
    bool use_seed = false;
    if (p0) {
        BVG_CUDA_TRY(cudaMemcpyAsync(g->s.p0, p0, (size_t)g->n * kb * sizeof(float), cudaMemcpyDeviceToDevice, st));
        p0_dev = g->s.p0;
    } else if (seeds && kb == 1) {
        BVG_CUDA_TRY(cudaMemsetAsync(g->s.p0, 0, (size_t)g->n * sizeof(float), st));
        BVG_CUDA_TRY(cudaMemcpyAsync(g->s.p0 + seeds[0], &kOne, sizeof(float), cudaMemcpyHostToDevice, st));
        p0_dev = g->s.p0;
    } else if (seeds) {
        BVG_CUDA_TRY(cudaMemcpyAsync(g->s.seed, seeds, (size_t)kb * sizeof(int64_t), cudaMemcpyHostToDevice, st));
        use_seed = true;
    }
    PrArgs base{};
    base.p0 = p0_dev;
    base.ldp0 = kb;
    base.seed = use_seed ? g->s.seed : nullptr;
    base.inv_outdeg = g->inv_outdeg;
    base.ldq = kb;
    base.st = pst;
    base.partial = g->s.partial;
    base.counter = g->s.counter;
    base.gcounter = g->s.counter + 1;
    base.tile_counter = g->s.counter + 1 + max_grid(g) / kPrGroup + 1;
    base.gpartial = g->s.gpartial;
    base.alpha = (float)(1.0 - damping);
    base.dangling_uniform = dangling;
    base.k = k;
    // start: q[0] = p_init / p0 / the seeds / uniform, scalars into sc[0]
    {
        PrArgs pa = base;
        pa.q_new = g->s.q[0];
        pa.sc_new = g->s.sc[0];
        const float* start = p_init ? p_init : p0_dev;
        BVG_KV_CASES(launch_pr_init, g, start, kb, pa, st);
    }
    // A chunk of kChunk updates (even, so it starts on parity 0 every time)
    // is captured once per configuration and replayed; the device state makes
    // updates past convergence or max_iter return at once.
    constexpr int kChunk = 8;
    const bool fused = use_fused(g, kb);
    const int key[7] = {kb, v, dangling, p0_dev != nullptr, use_points(g, kb) ? 1 : 0, fused ? 1 : 0, use_seed};
    if (g->s.pr_exec && (memcmp(key, g->s.pr_key, sizeof(key)) || g->s.pr_key_alpha != base.alpha ||
                         g->s.pr_key_ptr != g->s.q[0] || g->s.pr_key_z != g->s.z))
        drop_pr_graph(g);
    auto launch_update = [&](int par) {
        // update reading q[par], writing q[1 - par]
        PrArgs pa = base;
        pa.q_prev = g->s.q[par];
        pa.q_new = g->s.q[1 - par];
        pa.sc_prev = g->s.sc[par];
        pa.sc_new = g->s.sc[1 - par];
        if (fused) {  // one kernel per update, a programmatic dependent of the previous one
            const int64_t grid = (g->n + kFxT - 1) / kFxT;
            TraceScope ts(g, "pr_fused", st);
            launch_pdl(1, k_push_fx<1>, grid, kFxNT, st, fused_args(g, g->s.q[par], kb, g->inv_outdeg, nullptr, 0),
                       pa);
            return;
        }
        BVG_KV_CASES(launch_chain, g, g->s.q[par], kb, g->inv_outdeg, g->s.z, kb, pst, st);
        BVG_KV_CASES(launch_gather_pr, g, g->s.z, kb, pa, st);
    };
    PrState* hst = (PrState*)g->s.host_state;
    double* hres = (double*)((char*)g->s.host_state + sizeof(PrState));
    int launched = 0;
    int next_poll = std::min(max_iter, 2 * kChunk);
    double last_res = INFINITY;
    int last_res_iter = 0;
    if (!g->s.pr_exec) {
        Tracer* tr = g->tracer;
        const bool tr_on = tr && tr->on;
        if (tr) tr->on = false;
        cudaGraph_t graph = nullptr;
        // capture on a private stream (the caller's may be the legacy default
        // stream, which cannot be captured); capturing executes nothing
        if (!g->s.cap_stream) {
            cudaStream_t cs = nullptr;
            BVG_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            g->s.cap_stream = cs;
        }
        cudaStream_t cs = (cudaStream_t)g->s.cap_stream;
        BVG_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
        {
            cudaStream_t user = st;
            st = cs;  // launch_update launches on `st`
            for (int u = 0; u < kChunk; u++) launch_update(u & 1);
            st = user;
        }
        cudaError_t ce = cudaStreamEndCapture(cs, &graph);
        if (tr) tr->on = tr_on;
        if (ce != cudaSuccess) {
            cudaGetLastError();
            return fail(BVG_ERR_CUDA, "bvg_pagerank: capture failed: %s", cudaGetErrorString(ce));
        }
        cudaGraphExec_t exec = nullptr;
        ce = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            return fail(BVG_ERR_CUDA, "bvg_pagerank: instantiate failed: %s", cudaGetErrorString(ce));
        }
        g->s.pr_exec = exec;
        memcpy(g->s.pr_key, key, sizeof(key));
        g->s.pr_key_alpha = base.alpha;
        g->s.pr_key_ptr = g->s.q[0];
        g->s.pr_key_z = g->s.z;
    }
    for (;;) {
        while (launched < next_poll) {
            TraceScope ts(g, "pr_update_x8", st);
            BVG_CUDA_TRY(cudaGraphLaunch((cudaGraphExec_t)g->s.pr_exec, st));
            launched += kChunk;
        }
        BVG_CUDA_TRY(cudaGetLastError());
        // state and the residuals of both parities; the state says which is current
        BVG_CUDA_TRY(cudaMemcpyAsync(hst, pst, sizeof(PrState), cudaMemcpyDeviceToHost, st));
        BVG_CUDA_TRY(cudaMemcpyAsync(hres, g->s.sc[0] + 2 * kb, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        BVG_CUDA_TRY(cudaMemcpyAsync(hres + 32, g->s.sc[1] + 2 * kb, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        BVG_CUDA_TRY(cudaStreamSynchronize(st));
        if (hst->done || hst->iter >= max_iter) break;
        if (launched >= max_iter || hst->iter != launched)
            return fail(BVG_ERR_CUDA, "bvg_pagerank: device state did not advance (%d of %d updates)", hst->iter,
                        launched);
        // plan the next poll from the observed contraction of the residual
        const double* cur = hres + 32 * (hst->iter & 1);
        double r = 0;
        for (int c = 0; c < k; c++) r = std::max(r, cur[c]);
        int ahead = 8;
        if (std::isfinite(r) && r > 0 && tol > 0) {
            double rate = 1.0 - (1.0 - damping);
            if (std::isfinite(last_res) && hst->iter > last_res_iter && r < last_res)
                rate = std::max(rate, std::pow(r / last_res, 1.0 / (hst->iter - last_res_iter)));
            rate = std::min(rate, 0.999);
            double need = std::log(tol / r) / std::log(rate);
            ahead = (int)std::ceil(need);
            ahead = std::max(kChunk, std::min(ahead, 64));
        }
        last_res = r;
        last_res_iter = hst->iter;
        next_poll = std::min(max_iter, launched + ahead);
    }
    BVG_KV_CASES(launch_pr_final, g, pst, p_out, st);
    BVG_CUDA_TRY(cudaGetLastError());
    BVG_CUDA_TRY(cudaMemcpyAsync(hres, g->s.sc[hst->iter & 1] + 2 * kb, sizeof(double) * k, cudaMemcpyDeviceToHost,
                                 st));
    BVG_CUDA_TRY(cudaStreamSynchronize(st));
    if (iters_out) *iters_out = hst->iter;
    if (resid_out)
        for (int c = 0; c < k; c++) resid_out[c] = hres[c];
    if (hst->numeric) return fail(BVG_ERR_NUMERIC, "bvg_pagerank: non-finite value at update %d", hst->iter);
    if (!hst->done) return fail(BVG_ERR_NOT_CONVERGED, "bvg_pagerank: not converged after %d updates", hst->iter);
    return BVG_OK;
}

extern "C" int bvg_pagerank(const bvg_dev_graph* g, const bvg_pr_params* params, const float* p0,
                            const float* p_init, int32_t k, float* p_out, int32_t* iters_out, double* resid_out,
                            void* stream) {
    return pagerank_run(g, params, p0, nullptr, p_init, k, p_out, iters_out, resid_out, stream);
}

extern "C" int bvg_pagerank_seeds(const bvg_dev_graph* g, const bvg_pr_params* params, const int64_t* seeds,
                                  const float* p_init, int32_t k, float* p_out, int32_t* iters_out,
                                  double* resid_out, void* stream) {
    if (!seeds) return fail(BVG_ERR_INVALID_ARG, "bvg_pagerank_seeds: NULL seeds");
    return pagerank_run(g, params, nullptr, seeds, p_init, k, p_out, iters_out, resid_out, stream);
}

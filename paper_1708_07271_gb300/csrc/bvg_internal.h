// Internal structures of the BV-delta library (host and device sides).
#pragma once

#include <cstdint>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/bvg.h"

namespace bvg {

// Largest supported window and chain bound. The device layout packs the
// reference offset (1..31, 0 = none) in bits 0-4 of a row's meta byte and the
// chain depth in bits 5-6; a chain spans at most window * max_chain rows,
// which the encoder keeps within kMaxSpan so that one 32-bit mask holds a
// row's descendants (W = 7 with R = 3, W = 15 with R = 2, W = 31 with R = 1).
constexpr int kMaxWindow = 31;
constexpr int kMaxChain = 3;
constexpr int kMaxSpan = 32;
constexpr uint32_t kMetaOff = 31u;   // meta & kMetaOff: i - r_i (0 = no reference)
constexpr int kMetaDepthShift = 5;  // meta >> kMetaDepthShift: chain depth
// Halo of rows a tile needs beyond its own range to resolve reference
// chains locally.
constexpr int kHalo = kMaxSpan;
// Granularity (columns) of the interval carry-in lists of the column layout.
constexpr int kCarryTile = 128;
// Two tag bits on top of a 30-bit id.
constexpr uint32_t kIdBits = 30;
constexpr uint32_t kIdMask = (1u << kIdBits) - 1;
constexpr int64_t kMaxN = (int64_t)1 << kIdBits;

// Row-major word tags (difference row of row i):
//   kTagPlus   residual id j       (+x_j)
//   kTagMinus  dropped id j        (-x_j)
//   kTagIvS    interval start s    (followed by a kTagIvL word)
//   kTagIvL    interval length
// Column-major word tags (entries of column j, payload = source row k):
//   kTagPlus   +z_k, kTagMinus -z_k,
//   kTagIvS    an interval of row k starts at j  (D_j += z_k)
//   kTagIvL    an interval of row k ends before j (D_j -= z_k)
constexpr uint32_t kTagPlus = 0, kTagMinus = 1, kTagIvS = 2, kTagIvL = 3;
// Push gather: the first kGatherSlots entries of a column are read by every
// column's own straight-line code; the rest form tail items of at most
// kTailItem consecutive entries (start index | (count - 1) << 30), handed out
// to the CTA's threads evenly.
constexpr int kGatherSlots = 3;
constexpr int kTailItem = 4;
// Point columns (see build_point_cols): straight-line slots per column.
constexpr int kPointSlots = 4;
// Point columns with more tail entries than this are summed by a whole CTA.
constexpr uint32_t kLongColumn = 256;
inline uint32_t pack(uint32_t tag, uint32_t v) { return (tag << kIdBits) | v; }

void set_error(const char* fmt, ...);
int fail(int status, const char* fmt, ...);
// True when the allocation-failure hook (bvg_debug_fail_alloc) says that this
// allocation checkpoint fails; the caller then reports BVG_ERR_OOM.
bool inject_alloc_failure();

// Host copy of the device layout (built once per host graph, see layout.cpp).
struct HostLayout {
    std::vector<uint8_t> meta;
    std::vector<uint32_t> desc;
    std::vector<uint32_t> rowp, ent, colp, tent, carry_ptr, carry;
    std::vector<uint32_t> titem_ptr, titem;  // tail items of the column-major entries
    std::vector<float> inv_outdeg;
    bool built = false;
};

// Pull work items built from row-major difference rows (see build_pull_items).
struct PullItems {
    std::vector<uint32_t> pent, istart, irow, lrow, lint;
};
int build_pull_items(const uint32_t* rowp, const uint32_t* ent, int64_t n, int item, int min_len, PullItems& out,
                     bool only_if_worth);

// Point columns built from row-major difference rows (see build_point_cols).
struct PointCols {
    std::vector<uint32_t> colp, ent, titem_ptr, titem;
    std::vector<uint8_t> long_chunk;  // per kCarryTile columns: 1 if one has more than kPointSlots + kLongColumn entries
};
int build_point_cols(const uint32_t* rowp, const uint32_t* ent, int64_t n, PointCols& out);

}  // namespace bvg

struct bvg_host_graph {
    int64_t n = 0, m = 0;
    int32_t window = 7, max_chain = 3, min_interval = 4;
    std::vector<int32_t> ref;      // r_i or -1
    std::vector<uint8_t> depth;    // chain depth
    std::vector<uint32_t> outdeg;  // |v_i|
    // difference rows, row-major
    std::vector<int64_t> drop_ptr, res_ptr, iv_ptr;  // n+1 each
    std::vector<int32_t> drop, res, iv_s, iv_len;
    // gamma/delta bitstream
    std::vector<uint64_t> bits;
    int64_t nbits = 0;
    bvg_graph_stats stats{};
    mutable std::mutex layout_mu;
    mutable std::unique_ptr<bvg::HostLayout> layout;
};

namespace bvg {
// The encoder for a block of n rows over ncols columns (references among the
// block's rows); bvg_encode is encode_rows(n, n, ...).
int encode_rows(int64_t n, int64_t ncols, const int64_t* row_ptr, const int32_t* col_idx,
                const bvg_encode_params* params, bvg_host_graph** out);
int build_layout(const bvg_host_graph* hg, HostLayout& L);
int get_layout(const bvg_host_graph* hg, const HostLayout** out);
}  // namespace bvg

namespace bvg {

// Launch configuration of the product kernels (autotuned per graph and k).
struct LaunchCfg {
    int pull_tile = 512;        // rows per CTA of the pull's row pass
    int pull_prefix = -1;       // kept intervals: -1 keep only when worth a prefix (then use it), 0 keep and sum
                                // member by member, 1 keep and use the prefix of x
    int prefix_min_len = 32;    // pull: intervals at least this long stay (start, length); shorter ones are expanded
    int pull_item = 8;          // pull: entries per work item (4, 8 or 16)
    int gather_pdl = 1;         // launch the gather so it overlaps the chain kernel's tail
    int col_block = 32;         // widest column block of a product (power of two <= 32)
    int push_points = -1;       // x A gather over point columns: -1 every column block (default), 0 never (event
                                // columns), 1 always
    int push_fused = -1;        // x A for one right-hand side in one fused kernel (fused.cuh): -1 when the graph
                                // has locality (no tile reads rows outside its window), 0 never, 1 always
    int pull_fused = -1;        // A x^T for one right-hand side in one kernel (pull_fused.cuh): -1 or 1 whenever
                                // every tile's x window fits, 0 never
};

struct TuneInfo {
    int from_cache = 0;
    int candidates = 0;
    double push_us_default = 0, push_us_best = 0, pull_us_default = 0, pull_us_best = 0;
};

struct DevScratch {
    float* z = nullptr;                 // pushed weights, n x kcap (x A)
    float* q[2] = {nullptr, nullptr};   // PageRank iterates (unnormalised), n x pr_kcap
    double* sc[2] = {nullptr, nullptr}; // PageRank scalars per parity: [3][32] (1/S, dangling, resid)
    void* st = nullptr;                 // PageRank state (kernels.cuh PrState)
    int64_t* seed = nullptr;            // PageRank one-hot teleport nodes (32)
    double* partial = nullptr;          // per-CTA FP64 partial sums
    double* gpartial = nullptr;         // per group of CTAs (two-level reduction)
    unsigned int* counter = nullptr;    // [0]: groups finished; [1 + g]: CTAs of group g finished
    float* pre[4] = {nullptr, nullptr, nullptr, nullptr};  // prefix of x: L hi/lo ((n+1) x kcap), B hi/lo
    int64_t pre_kcap = 0;
    void* host_state = nullptr;         // pinned host copy of the state + residuals
    float* hx = nullptr;                // device staging for the host-buffer product
    float* hy = nullptr;
    int64_t kcap = 0;                   // columns the z buffer holds
    int64_t pr_kcap = 0;                // columns the PageRank buffers hold
    int64_t partial_cap = 0;            // doubles in `partial`
    int64_t stage_cap = 0;              // floats in hx / hy
    float* p0 = nullptr;                // PageRank teleport vectors (copy), n x pr_kcap
    // CUDA graph of a chunk of PageRank updates, and what it was built for
    void* pr_exec = nullptr;            // cudaGraphExec_t
    void* cap_stream = nullptr;         // private stream the update graph is captured on
    int pr_key[7] = {0, 0, 0, 0, 0, 0, 0}; // kb, v, dangling, has p0, point columns, fused update, seeds
    float pr_key_alpha = 0.f;
    const void* pr_key_ptr = nullptr;   // q[0] when captured
    const void* pr_key_z = nullptr;     // z when captured
    // warm-start features: degree temporaries (4 x n) and features + prediction (9 x n)
    float* feat_tmp = nullptr;
    int64_t feat_cap = 0;
    float* wfeat = nullptr;
    int64_t wfeat_cap = 0;
};

}  // namespace bvg

namespace bvg {
struct Tracer;  // api.cu
}

struct bvg_dev_graph {
    int64_t n = 0, m = 0;
    int device = 0;
    // row-major difference rows (A x^T)
    uint8_t* meta = nullptr;   // n: bits 0-2 reference offset (0 = none), bits 3-4 depth
    uint32_t* desc = nullptr;  // n: bit t set iff row i + t + 1 descends from row i
    uint32_t* rowp = nullptr;  // n+1 word offsets
    uint32_t* ent = nullptr;   // words
    int64_t nwords = 0;
    // column-major entries (x A)
    uint32_t* colp = nullptr;  // n+1
    uint32_t* tent = nullptr;
    int64_t ntent = 0;
    uint32_t* titem_ptr = nullptr;  // n + 1: tail items of column j are [titem_ptr[j], titem_ptr[j + 1])
    uint32_t* titem = nullptr;      // start in tent | (count - 1) << 30
    int64_t ntitem = 0;
    uint32_t* carry_ptr = nullptr;  // ceil(n / kCarryTile) + 1
    uint32_t* carry = nullptr;      // source rows of intervals open at a carry-tile start
    int64_t ncarry = 0;
    float* inv_outdeg = nullptr;    // 1/|v_i|, 0 for rows without successors
    double mean_interval = 0.0;     // mean interval length
    // pull work items: the difference rows with intervals shorter than
    // cfg.prefix_min_len expanded into single entries, cut into items of at
    // most cfg.pull_item entries; longer intervals kept as (start, length)
    uint32_t* pent = nullptr;       // expanded entries: id, bit 31 set for a dropped id
    uint32_t* istart = nullptr;     // nitems + 1: item k covers pent[istart[k], istart[k + 1])
    uint32_t* irow = nullptr;       // n + 1: items of row i are [irow[i], irow[i + 1])
    uint32_t* lrow = nullptr;       // n + 1: kept intervals of row i are [lrow[i], lrow[i + 1])
    uint32_t* lint = nullptr;       // 2 per kept interval: start, length
    int64_t npent = 0, nitems = 0, nlint = 0;
    float* part = nullptr;          // per item partial sums (compensated, rounded once) x part_kcap
    int64_t part_kcap = 0;
    int pull_built_item = 0, pull_built_minlen = 0, pull_built_auto = -1;  // parameters the items were built with
    int64_t pull_bytes = 0;                          // device bytes of the item arrays
    // point columns (x A): column-major entries with every interval member
    // expanded into a +z_k entry, so the gather needs no running interval sum;
    // tail items past the first kPointSlots entries. Built on first use.
    uint32_t* pcolp = nullptr;      // n + 1
    uint32_t* pcent = nullptr;      // kTagPlus / kTagMinus | source row
    uint32_t* ptitem_ptr = nullptr; // n + 1
    uint32_t* ptitem = nullptr;     // start in pcent | (count - 1) << 30
    uint8_t* plong = nullptr;       // per kCarryTile columns: holds a column longer than kPointSlots + kLongColumn
    int64_t npcent = 0, nptitem = 0, pcol_bytes = 0;
    // fused one-vector push (fused.cuh): per tile of its columns, 1 if an
    // entry or a carry source lies outside the tile's row window
    void* tile_win = nullptr;       // uint4 per tile: first and end row of its window, 1 if it reads a row outside
    uint16_t* tent16 = nullptr;     // fused kernel: event-column entries as window offsets (16-bit, see FxArgs)
    // one-vector pull (pull_fused.cuh): work items with every interval expanded, 16-bit window entries
    uint32_t* px_irow = nullptr;
    uint32_t* px_istart = nullptr;
    uint16_t* px_pent = nullptr;
    void* px_tile = nullptr;        // uint2 per tile of 1024 rows: its x window
    int px_ok = 0;                  // built, and every tile's window and items fit the kernel
    uint32_t* lane_cols = nullptr;  // fused kernel: 32 words per group of kCarryTile columns, each lane's 4 columns
    uint32_t* row_order = nullptr;  // fused kernel: the chain weights' row order, 256 words per 4 blocks of 256 rows
    int64_t row_groups = 0;
    int64_t fx_tiles = 0, fx_far_tiles = 0;
    unsigned int* err = nullptr;    // device word: a bounded wait ran out (read and cleared by bvg_device_check)
    int pcol_state = 0;             // 0 not built, 1 built, -1 too many entries (the event columns serve)
    std::vector<uint32_t> host_rowp, host_ent;       // the difference rows, to rebuild the items
    int64_t bytes = 0;
    bvg::LaunchCfg cfg;
    uint64_t fingerprint = 0;  // hash of the layout (autotune cache key)
    bvg::TuneInfo tune;
    bvg::DevScratch s;
    bvg::Tracer* tracer = nullptr;
};

namespace bvg {
// Point columns of a device graph (api.cu): built and copied on first use
// (synchronises `stream`); want_points: a kb-wide column block should read
// them; use_points: it does (they are built).
int ensure_points(bvg_dev_graph* g, void* stream);
bool want_points(const bvg_dev_graph* g, int kb);
bool use_points(const bvg_dev_graph* g, int kb);
// A vector argument of a device product: not NULL, 4-byte aligned, and device
// (or managed) memory of the graph's device; otherwise INVALID_ARG (api.cu).
int check_vec(const bvg_dev_graph* g, const void* p, const char* what);
// x A (one right-hand side, vectors contiguous) for the columns [col0, col1)
// only; BVG_ERR_UNSUPPORTED (nothing launched) unless the one-launch kernel
// serves g and the range is made of whole 1024-column tiles (api.cu).
int spmv_xA_columns(const bvg_dev_graph* g, const float* x, float* y, int64_t col0, int64_t col1, void* stream);
// The pull on a device graph view whose arrays the caller placed (api.cu).
int pull_view_product(const bvg_dev_graph* v, const float* x, float* y, int32_t k, int64_t ld, void* stream);
}  // namespace bvg

// Biclique decomposition (host; biclique.cpp): bicliques (S_r, C_r) as two
// CSR-like lists, residual edges by row.
struct bvg_biclique {
    int64_t n = 0, m = 0;
    std::vector<int64_t> s_ptr{0}, c_ptr{0}, r_ptr;
    std::vector<int32_t> s_idx, c_idx, r_col;
};

struct bvg_csr_graph {
    int64_t n = 0, m = 0;
    int device = 0;
    int64_t* rp = nullptr;  // CSR of A
    int32_t* ci = nullptr;
    int64_t* rpt = nullptr; // CSR of A^T
    int32_t* cit = nullptr;
    // rows longer than the hub threshold, summed by a whole CTA each
    int32_t* hub = nullptr;  // rows of A
    int32_t* hubt = nullptr; // rows of A^T
    int64_t nhub = 0, nhubt = 0;
    // cuSPARSE: 32-bit row offsets of A and A^T, values 1.0f, handle and
    // descriptors (created on the first cuSPARSE product), workspace
    int32_t* rp32 = nullptr;
    int32_t* rpt32 = nullptr;
    float* ones = nullptr;
    void* sp_handle = nullptr;
    void* sp_mat = nullptr;
    void* sp_matt = nullptr;
    void* sp_buf = nullptr;
    size_t sp_buf_bytes = 0;
};

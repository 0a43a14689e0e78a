// Streamed row blocks: y = M x^T for a matrix M whose compressed structure
// need not fit in device memory (the paper's own graphs reach 9e10 edges,
// Sec. 5, Table 1), and for many right-hand sides at once (the Online
// Matrix-Vector setting of Sec. 2: one pass over the structure serves every
// column of x).
//
// At creation the rows are cut into blocks of about equal edges; each block is
// encoded on its own (its references stay inside the block: the window of
// Sec. 4 looks only at the block's earlier rows), and only its pull image is
// kept, in page-locked host memory: reference offsets and chain depths,
// work items and expanded difference entries (every interval expanded, so no
// prefix of x is needed). A product walks the blocks in order through two
// device slots: a copy stream fills one slot while the pull kernels run on
// the other, the slot's next copy waiting for the kernels that read it. Each
// block serves all k columns of x before the next is copied. x A is the same
// stream built on A^T (left = 1).
#include <algorithm>
#include <climits>
#include <new>
#include <vector>

#include "kernels.cuh"

using namespace bvg;

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Block {
    int64_t r0 = 0, r1 = 0;           // rows [r0, r1) of M
    int64_t nitems = 0, npent = 0;
    int item = 8;                     // entries per work item
    size_t off_meta = 0, off_irow = 0, off_istart = 0, off_pent = 0, off_lrow = 0, bytes = 0;
    uint8_t* host = nullptr;          // page-locked image
    std::vector<int32_t> ref;         // references (global rows), for bvg_stream_get_refs
};

}  // namespace

struct bvg_stream {
    int64_t n_rows = 0, n_cols = 0, m = 0;
    int left = 0;
    int device = 0;
    std::vector<Block> blocks;
    size_t slot_bytes = 0;
    int64_t max_items = 0;
    uint8_t* slot[2] = {nullptr, nullptr};
    float* part = nullptr;            // item partial sums, max_items x 32
    uint32_t* lint = nullptr;         // no interval is kept whole: an empty list
    cudaStream_t copy = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr}, done[2] = {nullptr, nullptr};
    int64_t image_bytes = 0;          // sum of the blocks' images
};

namespace {

// The pull image of rows [r0, r1) of the CSR (ids in [0, ncols)).
int build_block(const int64_t* row_ptr, const int32_t* col, int64_t r0, int64_t r1, int64_t ncols,
                const bvg_encode_params* params, int item, Block& b) {
    const int64_t nb = r1 - r0, base = row_ptr[r0];
    std::vector<int64_t> rp(nb + 1);
    for (int64_t i = 0; i <= nb; i++) rp[i] = row_ptr[r0 + i] - base;
    bvg_host_graph* hg = nullptr;
    int rc = encode_rows(nb, ncols, rp.data(), col + base, params, &hg);
    if (rc) return rc;
    // row-major difference words (as the device layout stores them) -> work items
    std::vector<uint32_t> rowp(nb + 1, 0), ent;
    std::vector<uint8_t> meta(nb);
    b.ref.assign(nb, -1);
    for (int64_t i = 0; i < nb; i++) {
        const int off = hg->ref[i] >= 0 ? (int)(i - hg->ref[i]) : 0;
        meta[i] = (uint8_t)(off | (hg->depth[i] << kMetaDepthShift));
        b.ref[i] = hg->ref[i] >= 0 ? (int32_t)(r0 + hg->ref[i]) : -1;
        for (int64_t t = hg->drop_ptr[i]; t < hg->drop_ptr[i + 1]; t++) ent.push_back(pack(kTagMinus, hg->drop[t]));
        for (int64_t t = hg->res_ptr[i]; t < hg->res_ptr[i + 1]; t++) ent.push_back(pack(kTagPlus, hg->res[t]));
        for (int64_t t = hg->iv_ptr[i]; t < hg->iv_ptr[i + 1]; t++) {
            ent.push_back(pack(kTagIvS, hg->iv_s[t]));
            ent.push_back(pack(kTagIvL, hg->iv_len[t]));
        }
        rowp[i + 1] = (uint32_t)ent.size();
    }
    bvg_free_host(hg);
    PullItems P;
    if ((rc = build_pull_items(rowp.data(), ent.data(), nb, item, INT32_MAX, P, false))) return rc;
    b.r0 = r0;
    b.r1 = r1;
    b.item = item;
    b.nitems = (int64_t)P.istart.size() - 1;
    b.npent = (int64_t)P.pent.size();
    size_t o = 0;
    b.off_meta = o;
    o = align_up(o + nb);
    b.off_irow = o;
    o = align_up(o + (nb + 1) * 4);
    b.off_istart = o;
    o = align_up(o + P.istart.size() * 4);
    b.off_pent = o;
    o = align_up(o + std::max<size_t>(P.pent.size(), 1) * 4);
    b.off_lrow = o;
    o = align_up(o + (nb + 1) * 4);
    b.bytes = o;
    if (cudaMallocHost((void**)&b.host, b.bytes) != cudaSuccess) {
        cudaGetLastError();
        b.host = nullptr;
        return fail(BVG_ERR_OOM, "bvg_stream_create: page-locked host allocation failed");
    }
    std::copy(meta.begin(), meta.end(), b.host + b.off_meta);
    std::copy(P.irow.begin(), P.irow.end(), (uint32_t*)(b.host + b.off_irow));
    std::copy(P.istart.begin(), P.istart.end(), (uint32_t*)(b.host + b.off_istart));
    std::copy(P.pent.begin(), P.pent.end(), (uint32_t*)(b.host + b.off_pent));
    std::fill((uint32_t*)(b.host + b.off_lrow), (uint32_t*)(b.host + b.off_lrow) + nb + 1, 0u);
    return BVG_OK;
}

// A device graph view of the block image in a slot.
void view_of(const bvg_stream* s, const Block& b, const uint8_t* slot, bvg_dev_graph& v) {
    v.n = b.r1 - b.r0;
    v.m = 0;
    v.device = s->device;
    v.meta = (uint8_t*)(slot + b.off_meta);
    v.irow = (uint32_t*)(slot + b.off_irow);
    v.istart = (uint32_t*)(slot + b.off_istart);
    v.pent = (uint32_t*)(slot + b.off_pent);
    v.lrow = (uint32_t*)(slot + b.off_lrow);
    v.lint = s->lint;
    v.nitems = b.nitems;
    v.npent = b.npent;
    v.nlint = 0;
    v.part = s->part;
    v.part_kcap = 32;
    v.pull_built_item = b.item;
    v.tracer = nullptr;
}

}  // namespace

extern "C" void bvg_free_stream(bvg_stream* s) {
    if (!s) return;
    if (s->copy) cudaStreamSynchronize(s->copy);
    for (Block& b : s->blocks)
        if (b.host) cudaFreeHost(b.host);
    for (int t = 0; t < 2; t++) {
        if (s->slot[t]) cudaFree(s->slot[t]);
        if (s->copied[t]) cudaEventDestroy(s->copied[t]);
        if (s->done[t]) cudaEventDestroy(s->done[t]);
    }
    if (s->part) cudaFree(s->part);
    if (s->lint) cudaFree(s->lint);
    if (s->copy) cudaStreamDestroy(s->copy);
    delete s;
}

extern "C" int bvg_stream_create(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, int64_t budget_bytes,
                                 int32_t left, const bvg_encode_params* params, bvg_stream** out) {
    if (!out || n < 0 || !row_ptr || (n > 0 && row_ptr[n] > 0 && !col_idx) || budget_bytes <= 0 ||
        (left != 0 && left != 1))
        return fail(BVG_ERR_INVALID_ARG, "bvg_stream_create: bad argument");
    *out = nullptr;
    if (n >= kMaxN) return fail(BVG_ERR_UNSUPPORTED, "bvg_stream_create: n = %lld exceeds 2^30 - 1", (long long)n);
    const int64_t m = n > 0 ? row_ptr[n] : 0;
    bvg_stream* s = new (std::nothrow) bvg_stream();
    if (!s) return fail(BVG_ERR_OOM, "bvg_stream_create: host allocation failed");
    s->n_rows = s->n_cols = n;
    s->m = m;
    s->left = left;
    cudaGetDevice(&s->device);
    int rc = BVG_OK;
    try {
        // x A is the pull on A^T: transpose the CSR (rows sorted, no repeats)
        std::vector<int64_t> tp;
        std::vector<int32_t> tc;
        const int64_t* rp = row_ptr;
        const int32_t* ci = col_idx;
        if (left) {
            tp.assign(n + 1, 0);
            tc.resize((size_t)m);
            for (int64_t e = 0; e < m; e++) {
                if (col_idx[e] < 0 || col_idx[e] >= n) throw (int)BVG_ERR_BAD_GRAPH;
                tp[col_idx[e] + 1]++;
            }
            for (int64_t j = 0; j < n; j++) tp[j + 1] += tp[j];
            std::vector<int64_t> fill(tp.begin(), tp.end() - 1);
            for (int64_t i = 0; i < n; i++)
                for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++) tc[fill[col_idx[e]]++] = (int32_t)i;
            rp = tp.data();
            ci = tc.data();
        }
        // blocks: rows of about equal edges, each image at most half the budget
        // (two slots); an image that comes out larger is split in two
        const int item = 8;
        std::vector<std::pair<int64_t, int64_t>> todo;
        const int64_t target = std::max<int64_t>(1, budget_bytes / 2 / 6);  // edges per block (~6 bytes per edge)
        for (int64_t r = 0; r < n;) {
            int64_t r1 = r + 1;
            while (r1 < n && rp[r1 + 1] - rp[r] <= target) r1++;
            todo.push_back({r, r1});
            r = r1;
        }
        while (!todo.empty()) {
            auto [r0, r1] = todo.front();
            todo.erase(todo.begin());
            Block b;
            if ((rc = build_block(rp, ci, r0, r1, n, params, item, b))) throw rc;
            if (b.bytes > (size_t)budget_bytes / 2 && r1 - r0 > 1) {
                cudaFreeHost(b.host);
                const int64_t mid = r0 + (r1 - r0) / 2;
                todo.insert(todo.begin(), {r0, mid});
                todo.insert(todo.begin() + 1, {mid, r1});
                continue;
            }
            s->slot_bytes = std::max(s->slot_bytes, b.bytes);
            s->max_items = std::max(s->max_items, b.nitems);
            s->image_bytes += (int64_t)b.bytes;
            s->blocks.push_back(std::move(b));
        }
        if (s->slot_bytes > (size_t)budget_bytes / 2)
            throw fail(BVG_ERR_UNSUPPORTED, "bvg_stream_create: one row needs %zu bytes, over half the budget",
                       s->slot_bytes);
        cudaError_t e;
        for (int t = 0; t < 2; t++) {
            if (inject_alloc_failure() || cudaMalloc((void**)&s->slot[t], std::max<size_t>(s->slot_bytes, 16)) != cudaSuccess)
                throw fail(BVG_ERR_OOM, "bvg_stream_create: slot allocation failed");
            if ((e = cudaEventCreateWithFlags(&s->copied[t], cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&s->done[t], cudaEventDisableTiming)) != cudaSuccess)
                throw fail(BVG_ERR_CUDA, "bvg_stream_create: %s", cudaGetErrorString(e));
        }
        if (cudaMalloc((void**)&s->part, (size_t)std::max<int64_t>(s->max_items, 1) * 32 * sizeof(float)) !=
                cudaSuccess ||
            cudaMalloc((void**)&s->lint, 16) != cudaSuccess)
            throw fail(BVG_ERR_OOM, "bvg_stream_create: scratch allocation failed");
        if ((e = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking)) != cudaSuccess)
            throw fail(BVG_ERR_CUDA, "bvg_stream_create: %s", cudaGetErrorString(e));
        for (int t = 0; t < 2; t++) cudaEventRecord(s->done[t], s->copy);  // the slots start free
    } catch (int code) {
        cudaGetLastError();
        bvg_free_stream(s);
        return code == BVG_ERR_BAD_GRAPH ? fail(BVG_ERR_BAD_GRAPH, "bvg_stream_create: id out of range") : code;
    } catch (const std::bad_alloc&) {
        bvg_free_stream(s);
        return fail(BVG_ERR_OOM, "bvg_stream_create: host allocation failed");
    }
    *out = s;
    return BVG_OK;
}

extern "C" int bvg_stream_spmv(bvg_stream* s, const float* x, float* y, int32_t k, int64_t ld, void* stream) {
    if (!s || !x || !y) return fail(BVG_ERR_INVALID_ARG, "bvg_stream_spmv: NULL argument");
    if (k < 1 || ld < k) return fail(BVG_ERR_INVALID_ARG, "bvg_stream_spmv: need k >= 1 and ld >= k");
    if ((uintptr_t)x % 4 || (uintptr_t)y % 4) return fail(BVG_ERR_INVALID_ARG, "bvg_stream_spmv: misaligned");
    if (x == y) return fail(BVG_ERR_INVALID_ARG, "bvg_stream_spmv: x and y must not alias");
    for (const void* p : {(const void*)x, (const void*)y}) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess ||
            (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != s->device) {
            cudaGetLastError();
            return fail(BVG_ERR_INVALID_ARG, "bvg_stream_spmv: x and y must be memory of device %d", s->device);
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    for (size_t bi = 0; bi < s->blocks.size(); bi++) {
        const Block& b = s->blocks[bi];
        const int t = (int)(bi & 1);
        // copy the image once the kernels that read this slot last are done
        BVG_CUDA_TRY(cudaStreamWaitEvent(s->copy, s->done[t], 0));
        BVG_CUDA_TRY(cudaMemcpyAsync(s->slot[t], b.host, b.bytes, cudaMemcpyHostToDevice, s->copy));
        BVG_CUDA_TRY(cudaEventRecord(s->copied[t], s->copy));
        BVG_CUDA_TRY(cudaStreamWaitEvent(st, s->copied[t], 0));
        bvg_dev_graph v;
        view_of(s, b, s->slot[t], v);
        int rc = pull_view_product(&v, x, y + b.r0 * ld, k, ld, stream);
        if (rc) return rc;
        BVG_CUDA_TRY(cudaEventRecord(s->done[t], st));
    }
    return BVG_OK;
}

extern "C" int bvg_stream_info(const bvg_stream* s, bvg_stream_info_t* out) {
    if (!s || !out) return fail(BVG_ERR_INVALID_ARG, "bvg_stream_info: NULL argument");
    out->n = s->n_rows;
    out->m = s->m;
    out->left = s->left;
    out->blocks = (int64_t)s->blocks.size();
    out->slot_bytes = (int64_t)s->slot_bytes;
    out->image_bytes = s->image_bytes;
    return BVG_OK;
}

extern "C" int bvg_stream_get_refs(const bvg_stream* s, int32_t* ref) {
    if (!s || !ref) return fail(BVG_ERR_INVALID_ARG, "bvg_stream_get_refs: NULL argument");
    for (const Block& b : s->blocks) std::copy(b.ref.begin(), b.ref.end(), ref + b.r0);
    return BVG_OK;
}

/*
 * bvg.h -- C ABI of the BV-delta adjacency-product library for GB300 (sm_103a).
 *
 * The library computes y = A x^T and y = x A for a binary adjacency matrix A
 * directly on a reference/difference ("BV-delta") representation of A, and
 * PageRank on top of x A (Francisco, Gagie, Ladra, Navarro, "Exploiting
 * Computation-Friendly Graph Compression Methods for Adjacency-Matrix
 * Multiplication", Sec. 3-5).
 *
 * Representation (Sec. 4): row i of A is v_i; a reference r_i < i within a
 * window of W rows is chosen for each row (or none, the sentinel v_0 = 0),
 * and the difference row a'_i = v_i - v_{r_i} is stored: ids of v_{r_i}
 * missing from v_i (dropped, -1 entries), and ids added to it, split into
 * intervals (runs of >= min_interval consecutive ids) and residual ids.
 * Chains of references are at most max_chain long.
 *
 * Conventions for every call:
 *   - Return value: BVG_OK (0) or a negative bvg_status. No exception or
 *     abort crosses the ABI. bvg_last_error() gives a one-line reason for the
 *     last failure on the calling thread.
 *   - Ids are 0-based; n < 2^30 (two tag bits of a 32-bit word are used by
 *     the device layout).
 *   - Vectors with k right-hand sides are row-major n x k FP32 with leading
 *     dimension ld >= k (element (i, c) at ptr[i * ld + c]); device pointers
 *     must be 4-byte aligned, and 16-byte aligned with ld % 4 == 0 to use
 *     128-bit loads (otherwise narrower loads are used).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Device calls are asynchronous on that stream unless stated.
 *   - The caller owns every vector buffer; the library owns handles and their
 *     device memory and frees them only in bvg_free_*().
 *   - Handles are immutable after creation (bvg_autotune only updates the
 *     launch configuration stored in it); concurrent calls that use one
 *     handle must use one stream, since a handle holds scratch buffers.
 */
#ifndef BVG_H
#define BVG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BVG_OK = 0,
    BVG_ERR_INVALID_ARG = -1,   /* NULL or out-of-range argument, misaligned pointer */
    BVG_ERR_BAD_GRAPH = -2,     /* CSR not sorted, duplicate or out-of-range ids */
    BVG_ERR_OOM = -3,           /* host or device allocation failed */
    BVG_ERR_CUDA = -4,          /* a CUDA runtime call failed */
    BVG_ERR_NOT_CONVERGED = -5, /* PageRank hit max_iter; outputs hold the last iterate */
    BVG_ERR_NUMERIC = -6,       /* NaN/Inf met (e.g. in a PageRank iterate) */
    BVG_ERR_TIMEOUT = -7,       /* a bounded device wait ran out */
    BVG_ERR_CORRUPT = -8,       /* bitstream fails to decode */
    BVG_ERR_UNSUPPORTED = -9    /* size or option outside what the library supports */
} bvg_status;

typedef struct bvg_host_graph bvg_host_graph; /* host encoding: refs, difference rows, bitstream */
typedef struct bvg_dev_graph bvg_dev_graph;   /* device-resident BV-delta layout + scratch */
typedef struct bvg_csr_graph bvg_csr_graph;   /* device CSR of A and of A^T (plain baseline) */
typedef struct bvg_batch bvg_batch;           /* many device graphs for one persistent launch */
typedef struct bvg_mlp bvg_mlp;               /* warm-start network 6 -> 64 -> 64 -> 1 */

/* Encoder parameters (Sec. 4: window W; chain bound and interval length are
 * this library's choices). Zero fields take the defaults shown. */
typedef struct {
    int32_t window;       /* W, candidates r in [i - W, i - 1]; default 7, max 31 */
    int32_t max_chain;    /* R, longest reference chain; default 3, max 3; W * R at most 32 (a chain then
                             spans at most 32 rows: one 32-bit descendant mask per row) */
    int32_t min_interval; /* shortest run stored as an interval; default 4 */
    int32_t threads;      /* host threads for the cost pass; 0 = hardware concurrency */
} bvg_encode_params;

/* Sizes of an encoding. nnz_diff is nnz(A') (Table 1's m'); words is what the
 * device layout stores per row: dropped + residual + 2 * intervals. */
typedef struct {
    int64_t n, m;
    int64_t dropped, added, residual, intervals, interval_members;
    int64_t nnz_diff, words, rows_with_ref;
    int64_t depth_hist[4];   /* rows per chain depth 0..3 */
    int64_t bitstream_bits;  /* size of the gamma/delta-coded bitstream */
    double bits_per_edge;    /* bitstream_bits / m */
    int64_t device_bytes;    /* structure bytes of the device layout (both orientations) */
} bvg_graph_stats;

/* PageRank parameters (Sec. 3, Eq. 1). alpha = 1 - damping is the teleport
 * probability. */
typedef struct {
    double damping;   /* 1 - alpha; default 0.85 when 0 */
    double tol_l1;    /* stop when ||p_t - p_{t-1}||_1 < tol_l1 in every column */
    int32_t max_iter; /* bound on the number of updates; default 1000 when 0 */
    int32_t dangling; /* mass of zero-out-degree rows: 0 = along p0, 1 = uniform */
} bvg_pr_params;

/* ---------------------------------------------------------------- host side */

/* Encodes the binary matrix given by CSR (row_ptr: n+1 entries, row_ptr[0] = 0,
 * nondecreasing; col_idx: row_ptr[n] ids, strictly increasing within a row,
 * 0 <= id < n). Chooses references (Sec. 4 window, Sec. 5 keep-raw rule:
 * a reference is kept only if it is strictly cheaper than the raw row and
 * |v_i - v_r| < |v_i|), splits each difference row, and writes the bitstream.
 * Host-only and synchronous; the inputs are copied. *out is owned by the
 * caller (bvg_free_host). Errors: INVALID_ARG, BAD_GRAPH, UNSUPPORTED, OOM. */
int bvg_encode(int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
               const bvg_encode_params* params, bvg_host_graph** out);

/* Decodes the bitstream of `g` back into CSR (each row rebuilt from its
 * reference row and difference, Sec. 4). row_ptr (n+1) and col_idx (m) are
 * caller-allocated host arrays. decode(encode(A)) == A bit for bit.
 * Errors: INVALID_ARG, CORRUPT. */
int bvg_decode(const bvg_host_graph* g, int64_t* row_ptr, int32_t* col_idx);

/* The encoding's bitstream (the Sec. 4 representation; the paper fixes no
 * codes, this library writes gamma-coded reference offsets, copy blocks,
 * interval and residual counts, and delta-coded gaps), most significant bit
 * first in 64-bit words.
 * *nbits gets its length; if words != NULL the first ceil(nbits / 64) words
 * are copied there (cap_words at least that, else INVALID_ARG). Host only.
 * Errors: INVALID_ARG. */
int bvg_bitstream_get(const bvg_host_graph* g, uint64_t* words, int64_t cap_words, int64_t* nbits);

/* Decodes a caller-provided bitstream of n rows and m edges, written with
 * the window and minimum interval length of `params` (NULL = defaults), into
 * caller arrays row_ptr[n + 1] and col_idx[m]. Every count, offset and id is
 * checked against n, m, the window and the rows decoded so far before use:
 * a damaged or truncated stream returns BVG_ERR_CORRUPT and never reads or
 * writes outside the given buffers. Host only. Errors: INVALID_ARG,
 * UNSUPPORTED, CORRUPT, OOM. */
int bvg_decode_bits(int64_t n, int64_t m, const bvg_encode_params* params, const uint64_t* words, int64_t nbits,
                    int64_t* row_ptr, int32_t* col_idx);

/* Testing hook (the paper has no counterpart): after `after` further
 * allocation checkpoints, the next one fails once, as if the host or device
 * allocator had run out, and the call that reached it returns BVG_ERR_OOM
 * after releasing what it had allocated. Checkpoints: the start of
 * bvg_encode's allocations and every device allocation of bvg_upload and
 * the products. after < 0 disables the hook (the default). Always BVG_OK. */
int bvg_debug_fail_alloc(int64_t after);

/* Fills *out with the sizes of the encoding (Sec. 4's split of the
 * difference rows; nnz_diff is Table 1's m'). Host only. Errors:
 * INVALID_ARG. */
int bvg_stats(const bvg_host_graph* g, bvg_graph_stats* out);

/* Copies the reference vector (Sec. 4's r_i, or -1 for none; n entries)
 * and, if depth != NULL, the chain depth of every row, into caller host
 * arrays. Errors: INVALID_ARG. */
int bvg_get_refs(const bvg_host_graph* g, int32_t* ref, int32_t* depth);

/* Number of rows n and edges m of an encoding. Errors: INVALID_ARG. */
int bvg_host_size(const bvg_host_graph* g, int64_t* n, int64_t* m);

/* Read-only host view of the device layout that bvg_upload copies to the GPU
 * (built once per host graph and cached in it; the pointers stay valid until
 * bvg_free_host). Row-major words carry two tag bits above a 30-bit id:
 * 0 residual id (+1), 1 dropped id (-1), 2 interval start (next word: 3 |
 * length). Column-major entries carry the source row with tags 0 (+1 at this
 * column), 1 (-1), 2 (an interval of that row starts here), 3 (an interval
 * of that row ended just before this column). carry[carry_ptr[t] ..
 * carry_ptr[t+1]) lists the rows of intervals [s, e) with
 * s < t * carry_tile_cols <= e. meta[i] = (i - r_i, or 0) | depth_i << 5.
 * Tail items: column j's entries past its first 3 in runs of at most 4,
 * items [titem_ptr[j], titem_ptr[j+1]), each item = start index into the
 * column-major entries | (count - 1) << 30. */
typedef struct {
    int64_t n, words, col_entries, carry_tiles, carry_entries, carry_tile_cols;
    const uint8_t* meta;
    const uint32_t* desc; /* bit t: row i + t + 1 descends from row i (its chain passes through i) */
    const uint32_t* rowp;
    const uint32_t* ent;
    const uint32_t* colp;
    const uint32_t* tent;
    const uint32_t* carry_ptr;
    const uint32_t* carry;
    const float* inv_outdeg;
    int64_t tail_items;
    const uint32_t* titem_ptr;
    const uint32_t* titem;
} bvg_layout_view;
/* Fills *out; the arrays belong to g. Errors: INVALID_ARG, OOM (building the
 * layout), UNSUPPORTED (2^32 words or 2^30 column entries or more). */
int bvg_layout_view_get(const bvg_host_graph* g, bvg_layout_view* out);

/* -------------------------------------------------------------- device side */

/* The pull's work items, on the host (no GPU needed): each row's difference
 * row with the intervals shorter than min_len expanded into single entries
 * (a dropped id has bit 31 set), cut into items of at most `item` entries;
 * intervals at least min_len long kept as (start, length) pairs. Sizes first,
 * then the arrays into caller buffers: pent[entries], istart[items + 1]
 * (item k covers pent[istart[k], istart[k + 1])), irow[n + 1] (items of row
 * i: [irow[i], irow[i + 1])), lrow[n + 1] and lint[2 * intervals] (start,
 * length). bvg_upload builds the same arrays for the launch configuration's
 * pull_item and prefix_min_len. Errors: INVALID_ARG, OOM, UNSUPPORTED. */
int bvg_pull_items_size(const bvg_host_graph* g, int32_t item, int32_t min_len, int64_t* entries, int64_t* items,
                        int64_t* intervals);
int bvg_pull_items_fill(const bvg_host_graph* g, int32_t item, int32_t min_len, uint32_t* pent, uint32_t* istart,
                        uint32_t* irow, uint32_t* lrow, uint32_t* lint);

/* The push's point columns, on the host (no GPU needed): for every column j,
 * the source rows k of the nonzeros of column j of A' (Proposition 1's
 * difference matrix), in increasing k, as 32-bit words: tag (two high bits)
 * 0 for +1 (a residual id or a member of an interval of row k), 1 for -1 (a
 * dropped id), over the 30-bit row k. Every interval member is listed, so
 * y_j = sum of +-z_k over column j alone (no running interval sum).
 * colp[n + 1]: column j is ent[colp[j], colp[j + 1]). Tail items: the
 * entries of column j past its first 4, in runs of at most 4, items
 * [titem_ptr[j], titem_ptr[j + 1]), each item = start index | (count - 1)
 * << 30. Sizes first, then the arrays into caller buffers. The x A product
 * builds the same arrays on the device the first time a launch uses them.
 * Errors: INVALID_ARG, OOM, UNSUPPORTED (2^30 entries or more). */
int bvg_point_cols_size(const bvg_host_graph* g, int64_t* entries, int64_t* tail_items);
int bvg_point_cols_fill(const bvg_host_graph* g, uint32_t* colp, uint32_t* ent, uint32_t* titem_ptr, uint32_t* titem);

/* Builds the device layout of `g` (Sec. 4's difference rows: row-major for
 * A x^T, the same entries grouped by column for x A, per-row reference
 * offsets and chain depths, 1/outdeg for Eq. (1)) and copies it to the
 * current device on `stream`.
 * Also allocates the scratch of one-column products. The first product with
 * a wider column block grows that scratch, and the first x A with a column
 * block of 4 or more (under the default launch configuration) builds the
 * point columns (bvg_point_cols_size) and synchronises its stream; a caller
 * that must not allocate later makes one such call first, or uses
 * bvg_spmv_xA_noalloc. The host graph may be freed after this returns. *out
 * is owned by the caller (bvg_free_dev). Errors: INVALID_ARG, OOM, CUDA. */
int bvg_upload(const bvg_host_graph* g, void* stream, bvg_dev_graph** out);

/* y = A x^T (pull, Sec. 4): y_i = y_{r_i} + sum_j A'_ij x_j.
 * One right-hand side (a column block of width 1), by default: one launch
 * per product where every tile of 1024 rows fits it (the columns its rows'
 * entries reference, and those of the 32 rows before it, span at most 1792
 * ids; at most 2048 work items; no interval kept whole): x of the tile's
 * column window, the work items' sums, the row sums and the chains in shared
 * memory, with exact 64-bit fixed-point sums (y_i is the exact sum rounded
 * once to FP32) where the window's x spans few enough binades, compensated
 * sums otherwise (launch configuration pull_fused).
 * Otherwise: the row sums sum_j A'_ij x_j are formed per work item
 * (bvg_pull_items_size), then each row tile adds its rows' partials and
 * resolves the chains in shared memory (a row with more than 32 items, a hub
 * of a power-law graph, is summed by the whole tile's threads).
 * x, y: device n x k, leading dimension ld. Asynchronous. Errors:
 * INVALID_ARG, OOM (first call with a wider column block), CUDA. */
int bvg_spmv_Ax(const bvg_dev_graph* g, const float* x, float* y, int32_t k, int64_t ld, void* stream);

/* y = x A (push, Proposition 1 read for the left product): z_k = sum of x_i
 * over rows whose chain passes through k (x pushed down the reference chains
 * in reverse level order), then y = sum_k z_k a'_k, gathered per column with
 * no atomics (deterministic).
 * One right-hand side (a column block of width 1): by default one launch
 * computes, per tile of 1024 columns, the chain weights of the tile's row
 * window and the gather in shared memory, with exact 64-bit fixed-point sums
 * (y_j is the exact sum rounded once to FP32) where the tile's x spans few
 * enough binades, compensated sums otherwise; it serves graphs in which no
 * tile reads a row outside its window (launch configuration push_fused;
 * otherwise the two launches below). A timed-out internal copy sets the
 * graph's error word (bvg_device_check) and leaves NaN in y.
 * Wider column blocks: the chain launch, then the gather over the point
 * columns (bvg_point_cols_size) or the event columns (intervals as start /
 * end events and a running sum across columns, bvg_layout_view), as
 * push_points says; if the point columns cannot be built (2^30 entries or
 * more) the event columns serve. x, y: device n x k. Asynchronous. Errors:
 * INVALID_ARG, OOM, CUDA. */
int bvg_spmv_xA(const bvg_dev_graph* g, const float* x, float* y, int32_t k, int64_t ld, void* stream);

/* Same product as bvg_spmv_xA, for callers that must not allocate device
 * memory after set-up (a caller whose memory is owned by another allocator's
 * pool, a latency-critical loop that cannot afford cudaMalloc's implicit
 * synchronisation, an embedder that fixes the library's footprint at load
 * time). The paper has no counterpart: this is a property of this library.
 * It allocates nothing: the pushed weights live in a fixed 16 MiB device
 * array (4,194,304 floats) compiled into the library, which every GPU that
 * loads the library holds until the process exits. Requires n <= 4,194,304;
 * right-hand sides are processed in column blocks of at most
 * min(32, 4194304 / n); a larger n returns BVG_ERR_UNSUPPORTED. The first
 * call on each device looks up that array's device address (host-side, with
 * that device current) and caches it: make that first call before any stream
 * capture. Every call on a device shares the one array and each call
 * overwrites the part it uses before reading it, so nothing carries over;
 * calls that may overlap on the GPU (different streams, or in flight
 * together) race on it and must be serialised by the caller. x, y: device
 * n x k, leading dimension ld. Asynchronous on `stream`. Errors:
 * INVALID_ARG, UNSUPPORTED, CUDA. */
int bvg_spmv_xA_noalloc(const bvg_dev_graph* g, const float* x, float* y, int32_t k, int64_t ld, void* stream);

/* Reports a bounded device wait that ran out in an earlier launch on this
 * graph (the fused x A kernel waits for its TMA copies at most about 2 s and
 * then marks the graph and writes NaN outputs rather than hang): synchronises
 * `stream`, returns BVG_ERR_TIMEOUT (and clears the mark) if one did, else
 * BVG_OK. The paper has no counterpart. Errors: INVALID_ARG, TIMEOUT, CUDA. */
int bvg_device_check(const bvg_dev_graph* g, void* stream);

/* Same as bvg_spmv_xA (Proposition 1 read for the left product) with x and
 * y in HOST memory (page-locked, which copies fastest, or pageable), n x k,
 * ld == k: copies x to device scratch, runs the product, copies y back, and
 * synchronises `stream` before returning. The caller keeps both buffers.
 * Errors: INVALID_ARG (also when x and y alias), OOM, CUDA. */
int bvg_spmv_xA_host(const bvg_dev_graph* g, const float* x_host, float* y_host, int32_t k, void* stream);

/* PageRank by power iteration, Eq. (1): p_t = alpha p0 + (1 - alpha) p_{t-1} M,
 * M = D^-1 A, for k teleport vectors at once (k = 1, 2, 4, 8, 16 or 32, else
 * UNSUPPORTED; columns of p0, device n x k; NULL = uniform 1/n, then k must
 * be 1). p_init (device n x k or NULL =
 * start from p0) is the starting iterate. Iterates are FP32; the dangling
 * mass, the normalisation sum and the L1 change are FP64 on the device.
 * Stops after the first update with ||p_t - p_{t-1}||_1 < tol in every
 * column, or after max_iter updates. On return p_out (device n x k) holds the
 * last iterate normalised to sum 1 per column, *iters_out the number of
 * updates and resid_out[c] (host, k entries, may be NULL) the last L1 change.
 * Synchronises `stream`. Errors: INVALID_ARG, CUDA, NOT_CONVERGED (outputs
 * valid), NUMERIC. */
int bvg_pagerank(const bvg_dev_graph* g, const bvg_pr_params* params, const float* p0, const float* p_init,
                 int32_t k, float* p_out, int32_t* iters_out, double* resid_out, void* stream);

/* Personalised PageRank, Eq. (1) with one-hot teleport vectors: column c of
 * p0 is e_{seeds[c]} (1 at node seeds[c], 0 elsewhere), given by its node
 * instead of n x k floats. seeds: HOST array of k int64, each in [0, n),
 * read before the call returns (the caller keeps ownership). Same results as
 * bvg_pagerank with those dense vectors (the same arithmetic on the same
 * values); for k >= 2 the updates read no teleport vectors from memory.
 * p_init, k, p_out, iters_out, resid_out, stream and the synchronisation as
 * in bvg_pagerank. Errors: INVALID_ARG (NULL seeds, a seed outside [0, n),
 * or as bvg_pagerank), UNSUPPORTED (k), CUDA, NOT_CONVERGED (outputs valid),
 * NUMERIC. */
int bvg_pagerank_seeds(const bvg_dev_graph* g, const bvg_pr_params* params, const int64_t* seeds,
                       const float* p_init, int32_t k, float* p_out, int32_t* iters_out, double* resid_out,
                       void* stream);

/* ------------------------------------------------------ multi-graph batch */

/* A batch of device graphs whose products run in one grid: the chain step
 * of every graph in one kernel, the gather of every graph in a second one
 * (Proposition 1 applied to each graph independently), replayed from a
 * CUDA graph. The batch refers to the graphs' device layouts (no copy): the
 * graphs must outlive it. Graphs with n = 0 are accepted and skipped.
 * `stream` is unused (creation does no device work). Errors: INVALID_ARG,
 * OOM, CUDA. */
int bvg_batch_create(const bvg_dev_graph* const* gs, int32_t count, void* stream, bvg_batch** out);
/* Number of graphs, total rows and total edges of a batch. Errors:
 * INVALID_ARG. */
int bvg_batch_size(const bvg_batch* b, int32_t* count, int64_t* total_n, int64_t* total_m);
/* y_i = x_i A_i for every graph i (the push of Proposition 1 on each graph's
 * own encoding): xs[i], ys[i] (host arrays of `count`
 * DEVICE pointers) are row-major n_i x k with leading dimension k, 4-byte
 * aligned (16-byte alignment and k % 4 == 0 enable 128-bit accesses). The
 * pointer table is staged through pinned memory and copied on `stream`
 * ahead of the launches; the result of graph i is bit-identical to
 * bvg_spmv_xA on the same graph with the same buffers and launch
 * configuration (each graph's gather reads its event or point columns as its
 * configuration says; point columns not built yet are built first, which
 * synchronises `stream`). Calls on one batch are ordered among themselves
 * even across streams (a later call waits for the earlier one); the first
 * call with a larger k allocates. Asynchronous. Errors: INVALID_ARG, OOM,
 * CUDA. */
int bvg_batch_spmv_xA(bvg_batch* b, const float* const* xs, float* const* ys, int32_t k, void* stream);
/* Waits for the batch's last call, then frees it (not the graphs). */
void bvg_free_batch(bvg_batch* b);

/* ---------------------------------------------------- learned warm start */

/* The paper has no learned part: Eq. (1) converges to the same p from any
 * starting iterate, and this section only predicts a better start. A small
 * network 6 -> 64 -> 64 -> 1 (ReLU; weights rounded to BF16, FP32
 * accumulation, the 64 x 64 layer on tensor cores) maps node features to
 * yhat_i ~ n p_i; the start is p_init = max(yhat, 0.05) / sum(max(yhat, 0.05))
 * (n p*_i >= alpha under uniform teleport, so the floor only guards
 * against negative or NaN predictions).
 * Parameters: 4673 FP32 values laid out W1[64][6], b1[64], W2[64][64],
 * b2[64], w3[64], b3 (row-major, output index first). The handle owns them,
 * the Adam moments and a BF16 copy of the weights, on the device current at
 * bvg_mlp_create; every call must run with that device current. Calls on
 * one handle are serialised by the caller. */

/* New network with He-style initial weights drawn from `seed` (splitmix64 +
 * Box-Muller), zero biases. Errors: INVALID_ARG, OOM, CUDA. */
int bvg_mlp_create(uint64_t seed, bvg_mlp** out);
/* Number of parameters (4673); returns the count, not a status. */
int bvg_mlp_param_count(void);
/* Copies count (= 4673) host floats into the network, resets Adam, rounds
 * the BF16 copy. Synchronises the device. Errors: INVALID_ARG (NULL, or
 * count != 4673), CUDA. */
int bvg_mlp_set_params(bvg_mlp* net, const float* host, int64_t count);
/* Copies the FP32 parameters to host memory (count = 4673 floats).
 * Synchronises the device. Errors: INVALID_ARG, CUDA. */
int bvg_mlp_get_params(const bvg_mlp* net, float* host, int64_t count);
/* Node features of g into feat (device, n x 8 floats, 16-byte aligned):
 * log1p(in-degree), log1p(out-degree), reference-chain depth (Sec. 4),
 * fraction of the out-neighbours stored in intervals of the difference row
 * (Sec. 4), log1p(mean out-degree of the out-neighbours), log1p(weighted
 * in-degree sum_{j -> i} 1/outdeg(j)), 0, 0. The degrees come from two
 * compressed products: (1, 1/outdeg) A with k = 2, and A outdeg^T.
 * May grow the graph's scratch. Asynchronous on `stream`. Errors:
 * INVALID_ARG (NULL, feat not 16-byte aligned), OOM, CUDA. */
int bvg_features(const bvg_dev_graph* g, float* feat, void* stream);
/* yhat (device, n floats) for features feat (device n x 8, 16-byte aligned).
 * Asynchronous on `stream`. Errors: INVALID_ARG, CUDA. */
int bvg_mlp_predict(const bvg_mlp* net, const float* feat, int64_t n, float* yhat, void* stream);
/* Mean squared error of yhat against target (device, n floats) and its
 * gradient with respect to the FP32 parameters (rounding steps pass
 * gradients straight through). *loss (may be NULL) gets the loss; grad_host
 * (may be NULL, else 4673 host floats) the gradient, which also stays in the
 * handle for bvg_mlp_adam. Synchronises `stream`. Errors: INVALID_ARG, OOM,
 * CUDA. */
int bvg_mlp_grad(bvg_mlp* net, const float* feat, const float* target, int64_t n, double* loss,
                 float* grad_host, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with
 * the gradient of the last bvg_mlp_grad, then re-rounds the BF16 weights.
 * Asynchronous on `stream`. Errors: INVALID_ARG, CUDA. */
int bvg_mlp_adam(bvg_mlp* net, float lr, void* stream);
/* Trains on `count` graphs with known PageRank vectors p_star[i] (Eq. (1)'s
 * fixed points; the paper has no learned part) (device,
 * n_i floats): targets n p*, `epochs` passes over the nodes
 * in chunks of `batch` (>= 128) nodes, one Adam step per chunk. *loss (may
 * be NULL) gets the mean loss of the last pass. Allocates temporaries for
 * the features and frees them before returning. Synchronises `stream`.
 * Errors: INVALID_ARG, OOM, CUDA. */
int bvg_warmstart_train(bvg_mlp* net, const bvg_dev_graph* const* gs, const float* const* p_star, int32_t count,
                        int32_t epochs, float lr, int64_t batch, double* loss, void* stream);
/* p_init (device, n floats) = max(yhat, 0.05) normalised to sum 1 (FP64
 * sum; uniform 1/n where the sum is not finite) for g: a starting iterate
 * for bvg_pagerank (Eq. (1) reaches the same fixed point from any start; the
 * paper has no learned part). May grow the graph's scratch. Asynchronous on
 * `stream`. Errors: INVALID_ARG, OOM, CUDA. */
int bvg_warmstart_predict(const bvg_mlp* net, const bvg_dev_graph* g, float* p_init, void* stream);
void bvg_free_mlp(bvg_mlp* net);

/* Launch configuration of a device graph (what bvg_autotune chooses; the
 * results of every setting are the same up to the product tolerance). */
typedef struct {
    int32_t pull_tile;      /* rows per CTA of the pull's row pass: power of two in [64, 2048] (default 512) */
    int32_t pull_prefix;    /* pull: intervals of at least prefix_min_len ids: -1 kept whole (and summed from
                               the prefix of x) only when their members outnumber 2n, else expanded (default);
                               0 kept whole and summed member by member; 1 kept whole, summed from the prefix */
    int32_t prefix_min_len; /* pull: intervals at least this long stay (start, length) and are summed from the
                               prefix of x; shorter ones are expanded into work items (default 32) */
    int32_t gather_pdl;     /* 1: the push gather overlaps the chain kernel's tail (programmatic launch) */
    int32_t col_block;      /* widest column block of a product: power of two in [1, 32] (default 32) */
    int32_t pull_item;      /* pull: entries per work item, 4, 8 or 16 (default 8) */
    int32_t push_points;    /* push gather over the point columns: -1 for every column block (default), 0 never
                               (the event columns: intervals as start / end events and a running FP32 sum across
                               the tile, whose error is bounded relative to that running sum, not to the column's
                               own terms), 1 always */
    int32_t push_fused;     /* x A for one right-hand side in one kernel (exact fixed-point sums, TMA-staged
                               structure): -1 when no column tile reads rows outside its window (default), 0
                               never, 1 always */
    int32_t pull_fused;     /* A x^T for one right-hand side in one kernel (the x window of each tile of 1024
                               rows in shared memory, work items of at most 8 entries, exact fixed-point sums):
                               -1 or 1 whenever every tile's x window (at most 1792 columns) and work items (at
                               most 2048) fit the kernel (default -1), 0 never */
} bvg_launch_config;
/* The graph's configuration into *out. Errors: INVALID_ARG. */
int bvg_get_config(const bvg_dev_graph* g, bvg_launch_config* out);
/* Applies *in; a new pull_item or prefix_min_len rebuilds the pull's work
 * items. Errors: INVALID_ARG (a field outside the range its comment gives),
 * OOM, CUDA. */
int bvg_set_config(bvg_dev_graph* g, const bvg_launch_config* in);

/* Autotuner (the paper has no counterpart; its products and results are
 * those of Sec. 4 under every setting). Times the products of g with k
 * right-hand sides under each candidate launch configuration (CUDA events
 * on `stream`, median of 7 after 2 warm-up calls, warm caches): first the
 * push (x A) over the widest column block (the largest power of two
 * <= min(k, 32) and up to three halvings) times gather overlap on/off
 * times event or point columns, and for one
 * right-hand side the one-launch x A kernel too; then the pull (A x^T): for
 * one right-hand side the one-launch kernel where the graph fits it, and
 * the two-kernel pull over entries per work item {4, 8, 16} times rows per
 * CTA of the row pass {256, 512} times the length from which intervals stay
 * unexpanded (32; also 16 and "never" when the graph has intervals;
 * rebuilding the items is part of the search).
 * It applies the fastest choice to g (bvg_get_config shows it). With
 * cache_path != NULL it first looks the choice up in that JSON file under
 * the key "<device name>/sm<count>/<layout fingerprint>/k<k>" and, after a
 * search, stores it there (read-modify-write through a temporary file and a
 * rename; a missing or corrupt file starts a new cache). Allocates two
 * scratch n x k buffers for the search and frees them. Synchronises
 * `stream`. The results of every configuration agree up to the product
 * tolerance. Errors: INVALID_ARG, OOM, CUDA. */
int bvg_autotune(bvg_dev_graph* g, int32_t k, const char* cache_path, void* stream);
typedef struct {
    int32_t from_cache;      /* 1: the last bvg_autotune took the configuration from the cache */
    int32_t candidates;      /* configurations timed by the last bvg_autotune */
    double push_us_default;  /* x A before tuning, and with the chosen configuration (us) */
    double push_us_best;
    double pull_us_default;  /* A x^T likewise */
    double pull_us_best;
} bvg_autotune_info;
/* The last search's counts and timings. Errors: INVALID_ARG. */
int bvg_autotune_info_get(const bvg_dev_graph* g, bvg_autotune_info* out);
/* The cache key bvg_autotune uses for g and k (NUL-terminated, into buf of
 * cap bytes). Errors: INVALID_ARG (also when buf is too small), CUDA. */
int bvg_autotune_key(const bvg_dev_graph* g, int32_t k, char* buf, int32_t cap);
/* Host-only access to the cache file (no GPU needed): *found = 1 and *out
 * set when `key` is present; a missing or unreadable file gives *found = 0.
 * Errors: INVALID_ARG. */
int bvg_autotune_cache_lookup(const char* path, const char* key, bvg_launch_config* out, int32_t* found);
/* Inserts or replaces `key` (with the timings it was chosen by, in us).
 * Errors: INVALID_ARG (also when the file cannot be written or renamed into
 * place). */
int bvg_autotune_cache_store(const char* path, const char* key, const bvg_launch_config* cfg, double push_us,
                             double pull_us);

/* Number of rows n and edges m of a device graph. Errors: INVALID_ARG. */
int bvg_dev_size(const bvg_dev_graph* g, int64_t* n, int64_t* m);

/* Sizes of the device layout, for byte models: 32-bit words of the row-major
 * difference rows and of the column-major entries, carry-list entries
 * (interval sources open at each 128-column tile start), structure bytes. */
typedef struct {
    int64_t n, m, words, col_entries, carry_tiles, carry_entries, structure_bytes;
    int64_t pull_entries, pull_items, pull_intervals;  /* the pull's work items (see bvg_pull_items_size) */
    int64_t tail_items;                                /* the push gather's tail items (bvg_layout_view) */
    int64_t point_entries, point_tail_items;           /* the point columns (bvg_point_cols_size); 0 until built */
} bvg_layout_info;
/* Errors: INVALID_ARG. */
int bvg_dev_layout(const bvg_dev_graph* g, bvg_layout_info* out);

/* ------------------------------------------ biclique representation */

/* The second compressed format of the paper's final remarks (Sec. 6): the
 * edges are split into bicliques (S_r, C_r), every node of S_r pointing to
 * every node of C_r, stored as the two lists (|S_r| + |C_r| words for
 * |S_r| * |C_r| edges), plus residual edges. A x^T is then c_r = sum over C_r
 * of x, added to y_i for every i in S_r, plus the residual edges. The paper
 * cites an extraction method without describing it; bvg_biclique_encode uses
 * its own deterministic greedy miner (rows keyed by a min-hash of their
 * remaining successors, per pass; within a run of equal keys a biclique grows
 * row by row while |S| * |C| - (|S| + |C|) does not shrink, and is kept when
 * that saving is positive; bicliques with equal column sets are then merged).
 * Host only. */
typedef struct bvg_biclique bvg_biclique;  /* host decomposition */
typedef struct {
    int32_t passes;    /* min-hash passes; 0 = 8 */
    int32_t min_rows;  /* rows of a biclique at least; any value below 2 selects the default 2 */
    int32_t min_cols;  /* columns of a biclique at least; any value below 2 selects the default 3 */
    int32_t pad;
    uint64_t seed;     /* hash seed */
} bvg_biclique_params;
typedef struct {
    int64_t n, m;
    int64_t bicliques;       /* number of bicliques */
    int64_t s_total, c_total; /* sum |S_r|, sum |C_r| */
    int64_t residual;        /* residual edges */
    int64_t words;           /* s_total + c_total + residual */
    int64_t biclique_edges;  /* sum |S_r| * |C_r| (= m - residual) */
} bvg_biclique_info;
/* Decomposes the CSR of A (rows sorted, no repeats, ids in [0, n), n < 2^31;
 * copied). params may be NULL (defaults). *out is owned by the caller
 * (bvg_free_biclique). Synchronous. Errors: INVALID_ARG, OOM. */
int bvg_biclique_encode(int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
                        const bvg_biclique_params* params, bvg_biclique** out);
/* Sizes of the decomposition. Errors: INVALID_ARG. */
int bvg_biclique_stats(const bvg_biclique* b, bvg_biclique_info* out);
/* The decomposition into caller buffers sized from bvg_biclique_stats:
 * s_ptr[bicliques + 1], s_idx[s_total] (the rows of biclique r are
 * s_idx[s_ptr[r], s_ptr[r + 1]), increasing), c_ptr[bicliques + 1],
 * c_idx[c_total] (its columns, increasing), r_ptr[n + 1], r_col[residual]
 * (the residual edges of row i, increasing). The bicliques and the residual
 * edges are disjoint and together are exactly the edges of A. Errors:
 * INVALID_ARG. */
int bvg_biclique_get(const bvg_biclique* b, int64_t* s_ptr, int32_t* s_idx, int64_t* c_ptr, int32_t* c_idx,
                     int64_t* r_ptr, int32_t* r_col);
/* The lists a device product gathers from, into caller buffers: row_ptr2
 * [n + 1] and row_bic[s_total] (the bicliques whose S holds row i: for A x^T,
 * y_i adds their c_r), col_ptr2[n + 1] and col_bic[c_total] (the bicliques
 * whose C holds column j: for x A, y_j adds their sum over S), rt_ptr[n + 1]
 * and rt_row[residual] (the residual edges into column j, by source row).
 * Every list is increasing. Host only. Errors: INVALID_ARG. */
int bvg_biclique_gather_lists(const bvg_biclique* b, int64_t* row_ptr2, int32_t* row_bic, int64_t* col_ptr2,
                              int32_t* col_bic, int64_t* rt_ptr, int32_t* rt_row);
void bvg_free_biclique(bvg_biclique* b);

/* The biclique products on the device. bvg_biclique_upload copies a
 * decomposition and its gather lists to the current device (synchronising
 * `stream`); the decomposition may be freed afterwards. Errors: INVALID_ARG,
 * UNSUPPORTED (2^32 list entries or more), OOM, CUDA. */
typedef struct bvg_biclique_dev bvg_biclique_dev;
int bvg_biclique_upload(const bvg_biclique* b, void* stream, bvg_biclique_dev** out);
/* y = A x^T by the steps of Sec. 6: c_r = sum_{j in C_r} x_j for every
 * biclique, then y_i = sum of c_r over the bicliques whose S holds i, plus x_j
 * over row i's residual edges (a gather per row, no atomics; every sum
 * compensated and rounded once). x, y: device n x k, leading dimension ld.
 * The first call with a wider column block grows a per-biclique scratch
 * (synchronising `stream`); asynchronous otherwise. Errors: INVALID_ARG, OOM,
 * CUDA. */
int bvg_biclique_spmv_Ax(const bvg_biclique_dev* d, const float* x, float* y, int32_t k, int64_t ld, void* stream);
/* y = x A, the transpose of the same steps: d_r = sum_{i in S_r} x_i, then
 * y_j = sum of d_r over the bicliques whose C holds j, plus x_i over the
 * residual edges into column j. As bvg_biclique_spmv_Ax otherwise. Errors:
 * as bvg_biclique_spmv_Ax. */
int bvg_biclique_spmv_xA(const bvg_biclique_dev* d, const float* x, float* y, int32_t k, int64_t ld, void* stream);
void bvg_free_biclique_dev(bvg_biclique_dev* d);

/* ------------------------------------------------------------ streamed blocks */
/* y = M x^T for a matrix whose compressed structure need not fit in device
 * memory (the paper's graphs reach 9e10 edges, Sec. 5, Table 1), and for
 * many right-hand sides per pass over the structure (the Online
 * Matrix-Vector setting of Sec. 2). bvg_stream_create cuts the rows of M (M =
 * A, or A^T when left = 1, for x A) into blocks of about equal edges, encodes
 * each block on its own (references only among the block's rows, Sec. 4) and
 * keeps each block's pull image (reference offsets, chain depths, work items,
 * expanded difference entries) in page-locked host memory; no image exceeds
 * half of budget_bytes, and the device holds two of them plus item scratch
 * (max items x 32 floats). Host-side and synchronous; the CSR is copied.
 * Errors: INVALID_ARG, BAD_GRAPH, UNSUPPORTED (a single row's image over half
 * the budget), OOM, CUDA. */
typedef struct bvg_stream bvg_stream;
typedef struct {
    int64_t n, m;
    int32_t left, pad;
    int64_t blocks;       /* row blocks */
    int64_t slot_bytes;   /* device bytes of one slot (the largest image) */
    int64_t image_bytes;  /* page-locked bytes of all images */
} bvg_stream_info_t;
/* Creates the streamed encoding described above; *out is owned by the caller
 * (bvg_free_stream). Errors: INVALID_ARG, BAD_GRAPH, UNSUPPORTED, OOM, CUDA. */
int bvg_stream_create(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, int64_t budget_bytes, int32_t left,
                      const bvg_encode_params* params, bvg_stream** out);
/* y = M x^T (x A when the stream was created with left = 1; the pull of
 * Sec. 4 on each row block), x, y device n x k of leading dimension ld: the
 * blocks in order, each image copied on a
 * private copy stream into one of two device slots while the pull kernels of
 * the previous block run on `stream` (the slot's next copy waits for the
 * kernels that read it); every column of x is served before the next block
 * is copied. Asynchronous on `stream`; calls on one handle must be
 * serialised. Errors: INVALID_ARG (also x or y not memory of the handle's
 * device), CUDA. */
int bvg_stream_spmv(bvg_stream* s, const float* x, float* y, int32_t k, int64_t ld, void* stream);
/* Sizes of the streamed encoding. Errors: INVALID_ARG. */
int bvg_stream_info(const bvg_stream* s, bvg_stream_info_t* out);
/* The references of the block encodings (rows of M, -1 for none), n ints
 * into a caller host array. Errors: INVALID_ARG. */
int bvg_stream_get_refs(const bvg_stream* s, int32_t* ref);
void bvg_free_stream(bvg_stream* s);

/* --------------------------------------------------- plain CSR baseline */

/* Device CSR of A and of A^T built from a host CSR (same input rules as
 * bvg_encode), for the plain sparse product the compressed one is compared
 * with (Sec. 5 compares A' against A). *out is owned by the caller
 * (bvg_free_csr). Errors: INVALID_ARG, BAD_GRAPH, OOM, CUDA. */
int bvg_csr_upload(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, void* stream,
                   bvg_csr_graph** out);
/* y = A x^T over the CSR of A (a row per thread group, a hub row by a whole
 * CTA, no atomics). x, y: device n x k, leading dimension ld. Asynchronous.
 * Errors: INVALID_ARG, CUDA. */
int bvg_csr_spmv_Ax(const bvg_csr_graph* g, const float* x, float* y, int32_t k, int64_t ld, void* stream);
/* y = x A over the CSR of A^T (same kernel, transposed pattern). As
 * bvg_csr_spmv_Ax otherwise. Errors: INVALID_ARG, CUDA. */
int bvg_csr_spmv_xA(const bvg_csr_graph* g, const float* x, float* y, int32_t k, int64_t ld, void* stream);
/* The same two products by the vendor library (cusparseSpMV for one
 * right-hand side with ld = 1, cusparseSpMM on the row-major n x k block
 * otherwise; values 1.0f, 32-bit indices, the CSR of A^T for x A): the second
 * uncompressed baseline of the comparison of Sec. 5. The first call creates
 * the library handle and descriptors, and a call may grow a workspace
 * (synchronising `stream`). Asynchronous otherwise. Errors: INVALID_ARG,
 * UNSUPPORTED (2^31 edges or more), OOM, CUDA. */
int bvg_csr_cusparse_Ax(const bvg_csr_graph* g, const float* x, float* y, int32_t k, int64_t ld, void* stream);
int bvg_csr_cusparse_xA(const bvg_csr_graph* g, const float* x, float* y, int32_t k, int64_t ld, void* stream);

/* --------------------------------------------------- column blocks (Sec. 6) */

/* Products over A split into submatrices of consecutive columns, the split
 * that Sec. 6 proposes so that a reference need only match the part of a row
 * inside one block: A = sum_b A_b, where A_b holds A's entries in columns
 * [cuts[b], cuts[b+1]) and is encoded and uploaded on its own (n rows, the
 * same ids: bvg_encode of the column-restricted CSR, then bvg_upload), so
 * that each block chooses its own references. All blocks have the same n and
 * were uploaded on the same device.
 * cuts: host array of nblocks + 1 column bounds, cuts[0] = 0, cuts[nblocks]
 * = n, nondecreasing; block b must hold no entry outside its columns (not
 * checked: such entries are dropped from x A). scratch: device n x k (leading
 * dimension ld) owned by the caller, unused when nblocks = 1. x, y: device
 * n x k. Asynchronous; no allocation beyond what the blocks' own products
 * make. Errors: INVALID_ARG, and those of bvg_spmv_xA / bvg_spmv_Ax.
 *   x A:   block b's product goes to scratch, and its rows [cuts[b],
 *          cuts[b+1]) (the only nonzero ones) are copied into y; with one
 *          contiguous right-hand side (k = 1, ld = 1) and block bounds that
 *          are multiples of 1024 (or n), one launch computes every block's
 *          own column tiles into y when all blocks (at most 16) run the
 *          one-launch kernel, and otherwise each block that does computes
 *          just its own columns, into y;
 *   A x^T: y = sum_b A_b x^T, added in block order in FP32 (one rounding
 *          more per block). */
int bvg_spmv_xA_colblocks(const bvg_dev_graph* const* blocks, const int64_t* cuts, int32_t nblocks,
                          const float* x, float* y, float* scratch, int32_t k, int64_t ld, void* stream);
int bvg_spmv_Ax_colblocks(const bvg_dev_graph* const* blocks, int32_t nblocks, const float* x, float* y,
                          float* scratch, int32_t k, int64_t ld, void* stream);

/* -------------------------------------------------------------- tracing */

/* Per-kernel timing: while enabled, every kernel the library launches for
 * graph `g` is bracketed by two CUDA events on the launching stream. */
typedef struct {
    char name[32];     /* kernel family, e.g. "push_gather" */
    int64_t launches;  /* launches recorded since the last read */
    double total_ms;   /* sum of event-measured durations */
} bvg_trace_entry;

/* Turns tracing on (enable != 0) or off. Enabling allocates a pool of events
 * (host-side setup; call outside any stream capture). The paper has no
 * counterpart. Errors: INVALID_ARG, OOM, CUDA. */
int bvg_trace_enable(bvg_dev_graph* g, int enable);
/* Waits for the recorded events, aggregates them per kernel family into out
 * (at most cap entries; *count = families written) and clears the record.
 * Launches beyond the pool (65536 per read) are not recorded. Errors:
 * INVALID_ARG, CUDA. */
int bvg_trace_read(bvg_dev_graph* g, bvg_trace_entry* out, int32_t cap, int32_t* count);

/* ------------------------------------------------------------- lifetime */

/* Release a handle and the memory it owns (host, device and page-locked);
 * NULL is ignored. No call may use the handle afterwards. */
void bvg_free_host(bvg_host_graph* g);
void bvg_free_dev(bvg_dev_graph* g);
void bvg_free_csr(bvg_csr_graph* g);

/* Static description of a status code. */
const char* bvg_status_string(int status);
/* Reason for the last failure on this thread ("" if none). */
const char* bvg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* BVG_H */

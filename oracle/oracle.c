/*
 * ORACLE -- test infrastructure only.
 *
 * Plain, slow, obviously correct FP64 CPU implementation of what the
 * compressed adjacency product computes (Francisco, Gagie, Ladra, Navarro,
 * "Exploiting Computation-Friendly Graph Compression Methods for
 * Adjacency-Matrix Multiplication"). It shares no code with the CUDA
 * library: it derives the difference matrix A' from the CSR of A and a
 * reference vector r itself, by sorted-list merges, and never reads the
 * library's encoding. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.
 *
 * Conventions: rows/columns are 0-based; "no reference" is r_i = -1 and
 * plays the role of the paper's sentinel row v_0 = 0 (Sec. 4). Vectors with
 * k right-hand sides are row-major n x k.
 *
 * Functions and the passages they follow:
 *   oracle_csr_Ax / oracle_csr_xA   y = A x^T and y = x A by definition
 *                                   (Sec. 1; A_uv = 1 iff (u,v) in E, Sec. 3)
 *   oracle_choose_refs              reference choice within window W
 *                                   (Sec. 4) with the keep-raw rule of Sec. 5
 *   oracle_bv_Ax                    the sequential algorithm of Sec. 4:
 *                                   y_i = y_{r_i} + sum_j A'_ij x_j, i increasing
 *   oracle_bv_xA                    the same identity (Proposition 1) used
 *                                   for the left product: v_i is the sum of
 *                                   A' rows along its reference chain, so
 *                                   x A = sum_k z_k a'_k with z_k the sum of
 *                                   x over the rows whose chain contains k
 *   oracle_counts                   nnz(A') (Sec. 4-5, Table 1's m') and the
 *                                   interval/residual split of added entries
 *   oracle_pagerank                 power iteration, Eq. (1), M = D^-1 A (Sec. 3)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* y[i,:] = sum_j A_ij x[j,:] */
void oracle_csr_Ax(int64_t n, const int64_t* rp, const int32_t* ci, const double* x, int32_t k,
                   double* y) {
    for (int64_t i = 0; i < n; i++) {
        for (int32_t c = 0; c < k; c++) {
            double s = 0.0;
            for (int64_t e = rp[i]; e < rp[i + 1]; e++) s += x[(int64_t)ci[e] * k + c];
            y[i * k + c] = s;
        }
    }
}

/* y[j,:] = sum_i x[i,:] A_ij */
void oracle_csr_xA(int64_t n, const int64_t* rp, const int32_t* ci, const double* x, int32_t k,
                   double* y) {
    memset(y, 0, sizeof(double) * (size_t)(n * k));
    for (int64_t i = 0; i < n; i++)
        for (int64_t e = rp[i]; e < rp[i + 1]; e++)
            for (int32_t c = 0; c < k; c++) y[(int64_t)ci[e] * k + c] += x[i * k + c];
}

/* ---- the difference row a'_i = v_i - v_{r_i} ------------------------- */

/* Walks the merge of sorted rows v_i and v_r; calls back with (j, +1) for
 * j in v_i \ v_r and (j, -1) for j in v_r \ v_i. r < 0 means v_r = 0. */
typedef void (*diff_cb)(int32_t j, int sign, void* ctx);

static void diff_row(const int64_t* rp, const int32_t* ci, int64_t i, int64_t r, diff_cb cb,
                     void* ctx) {
    int64_t a = rp[i], ae = rp[i + 1];
    int64_t b = r >= 0 ? rp[r] : 0, be = r >= 0 ? rp[r + 1] : 0;
    while (a < ae || b < be) {
        if (b >= be || (a < ae && ci[a] < ci[b])) {
            cb(ci[a++], +1, ctx);
        } else if (a >= ae || ci[b] < ci[a]) {
            cb(ci[b++], -1, ctx);
        } else {
            a++;
            b++;
        }
    }
}

/* Counts of a difference row: dropped (-1 entries) and the added (+1)
 * entries split into maximal runs of consecutive ids; a run of length
 * >= lmin is an interval, shorter runs are residual ids. */
typedef struct {
    int64_t dropped, added, residual, intervals, interval_members;
    int32_t run_start, run_len, have_run, lmin;
} row_counts;

static void flush_run(row_counts* c) {
    if (c->have_run) {
        if (c->run_len >= c->lmin) {
            c->intervals += 1;
            c->interval_members += c->run_len;
        } else {
            c->residual += c->run_len;
        }
    }
    c->have_run = 0;
}

static void count_cb(int32_t j, int sign, void* ctx) {
    row_counts* c = (row_counts*)ctx;
    if (sign < 0) {
        c->dropped++;
        return;
    }
    c->added++;
    if (c->have_run && j == c->run_start + c->run_len) {
        c->run_len++;
    } else {
        flush_run(c);
        c->have_run = 1;
        c->run_start = j;
        c->run_len = 1;
    }
}

static row_counts row_diff_counts(const int64_t* rp, const int32_t* ci, int64_t i, int64_t r,
                                  int32_t lmin) {
    row_counts c;
    memset(&c, 0, sizeof(c));
    c.lmin = lmin;
    diff_row(rp, ci, i, r, count_cb, &c);
    flush_run(&c);
    return c;
}

/* Device-word cost of encoding row i against r: one word per dropped id,
 * one per residual id, two per interval. */
static int64_t row_cost(const row_counts* c) { return c->dropped + c->residual + 2 * c->intervals; }

/*
 * Reference choice. For row i the candidates are r in [max(0, i-W), i-1]
 * (r_i < i, Sec. 4) whose own reference chain is shorter than R (so that
 * every chain has at most R references). The chosen candidate minimises the
 * encoding cost (ties go to the nearest row); it is kept only if it costs
 * strictly less than encoding v_i alone and, following Sec. 5, only if
 * |v_i - v_r| < |v_i| (otherwise v_i is kept raw). ref[i] = -1 means none.
 * depth[i] (optional) receives the chain length of row i.
 */
void oracle_choose_refs(int64_t n, const int64_t* rp, const int32_t* ci, int32_t W, int32_t R,
                        int32_t lmin, int32_t* ref, int32_t* depth_out) {
    int32_t* depth = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; i++) {
        row_counts raw = row_diff_counts(rp, ci, i, -1, lmin);
        int64_t best_cost = -1, best_r = -1;
        int64_t best_nnz = 0;
        for (int64_t r = i - 1; r >= 0 && r >= i - W; r--) {
            if (depth[r] >= R) continue;
            row_counts c = row_diff_counts(rp, ci, i, r, lmin);
            int64_t cost = row_cost(&c);
            if (best_r < 0 || cost < best_cost) {
                best_cost = cost;
                best_r = r;
                best_nnz = c.dropped + c.added;
            }
        }
        int64_t deg = rp[i + 1] - rp[i];
        if (best_r >= 0 && best_cost < row_cost(&raw) && best_nnz < deg) {
            ref[i] = (int32_t)best_r;
            depth[i] = depth[best_r] + 1;
        } else {
            ref[i] = -1;
            depth[i] = 0;
        }
        if (depth_out) depth_out[i] = depth[i];
    }
    free(depth);
}

/* Totals over all rows for a given reference vector:
 * out[0] = dropped, out[1] = added, out[2] = residual ids, out[3] = intervals,
 * out[4] = interval members, out[5] = nnz(A') = dropped + added,
 * out[6] = device words = dropped + residual + 2 * intervals,
 * out[7] = rows with a reference. */
void oracle_counts(int64_t n, const int64_t* rp, const int32_t* ci, const int32_t* ref, int32_t lmin,
                   int64_t* out) {
    memset(out, 0, sizeof(int64_t) * 8);
    for (int64_t i = 0; i < n; i++) {
        row_counts c = row_diff_counts(rp, ci, i, ref[i], lmin);
        out[0] += c.dropped;
        out[1] += c.added;
        out[2] += c.residual;
        out[3] += c.intervals;
        out[4] += c.interval_members;
        out[5] += c.dropped + c.added;
        out[6] += row_cost(&c);
        out[7] += ref[i] >= 0;
    }
}

/* ---- products on A' -------------------------------------------------- */

typedef struct {
    const double* x;  /* gather source */
    double* acc;      /* k accumulators */
    int32_t k;
    int absval;       /* accumulate |A'_ij| |x_j| instead */
} gather_ctx;

static void gather_cb(int32_t j, int sign, void* p) {
    gather_ctx* g = (gather_ctx*)p;
    const double* xj = g->x + (int64_t)j * g->k;
    for (int32_t c = 0; c < g->k; c++) {
        if (g->absval) g->acc[c] += fabs(xj[c]);
        else g->acc[c] += sign > 0 ? xj[c] : -xj[c];
    }
}

/*
 * y = A x^T by the algorithm of Sec. 4: set y = 0 (and the sentinel
 * y_none = 0), then for i = 0..n-1 in increasing order
 *     y_i = y_{r_i} + sum_j A'_ij x_j,
 * where y_{r_i} was computed earlier because r_i < i.
 * With absval != 0 the same recursion accumulates |A'_ij| |x_j|, which is
 * the magnitude of every term the compressed formula adds into y_i (used as
 * the scale of the per-entry tolerance).
 */
void oracle_bv_Ax(int64_t n, const int64_t* rp, const int32_t* ci, const int32_t* ref,
                  const double* x, int32_t k, int absval, double* y) {
    double* acc = (double*)malloc(sizeof(double) * (size_t)k);
    for (int64_t i = 0; i < n; i++) {
        for (int32_t c = 0; c < k; c++) acc[c] = 0.0;
        gather_ctx g = {x, acc, k, absval};
        diff_row(rp, ci, i, ref[i], gather_cb, &g);
        for (int32_t c = 0; c < k; c++) {
            double w = ref[i] >= 0 ? y[(int64_t)ref[i] * k + c] : 0.0; /* w_i = y_{r_i} */
            y[i * k + c] = w + acc[c];
        }
    }
    free(acc);
}

typedef struct {
    const double* z;
    double* y;
    int64_t row;
    int32_t k;
    int absval;
} scatter_ctx;

static void scatter_cb(int32_t j, int sign, void* p) {
    scatter_ctx* s = (scatter_ctx*)p;
    const double* zr = s->z + s->row * s->k;
    double* yj = s->y + (int64_t)j * s->k;
    for (int32_t c = 0; c < s->k; c++) {
        if (s->absval) yj[c] += fabs(zr[c]);
        else yj[c] += sign > 0 ? zr[c] : -zr[c];
    }
}

/*
 * y = x A on the same A' and r. Since a'_i = v_i - v_{r_i}, row v_i is the
 * sum of the A' rows along its chain i, r_i, r_{r_i}, ... (Proposition 1
 * applied row by row), hence
 *     x A = sum_i x_i v_i = sum_k z_k a'_k,
 *     z_k = sum of x_i over the rows i whose chain passes through k.
 * z is formed by pushing each row's value to its reference in decreasing
 * row order (every row a reference points to has a smaller index, so a row
 * is complete before it is pushed). With absval != 0, |z| and |A'| are used
 * (z built from |x|), giving the term magnitudes for the tolerance.
 */
void oracle_bv_xA(int64_t n, const int64_t* rp, const int32_t* ci, const int32_t* ref,
                  const double* x, int32_t k, int absval, double* y) {
    double* z = (double*)malloc(sizeof(double) * (size_t)(n * k > 0 ? n * k : 1));
    for (int64_t t = 0; t < n * k; t++) z[t] = absval ? fabs(x[t]) : x[t];
    for (int64_t i = n - 1; i >= 0; i--)
        if (ref[i] >= 0)
            for (int32_t c = 0; c < k; c++) z[(int64_t)ref[i] * k + c] += z[i * k + c];
    memset(y, 0, sizeof(double) * (size_t)(n * k));
    for (int64_t i = 0; i < n; i++) {
        scatter_ctx s = {z, y, i, k, absval};
        diff_row(rp, ci, i, ref[i], scatter_cb, &s);
    }
    free(z);
}

/* z itself (the pushed weights), for inspection by tests. */
void oracle_chain_weights(int64_t n, const int32_t* ref, const double* x, int32_t k, double* z) {
    for (int64_t t = 0; t < n * k; t++) z[t] = x[t];
    for (int64_t i = n - 1; i >= 0; i--)
        if (ref[i] >= 0)
            for (int32_t c = 0; c < k; c++) z[(int64_t)ref[i] * k + c] += z[i * k + c];
}

/*
 * PageRank by power iteration, Eq. (1):
 *     p_t = alpha p_0 + (1 - alpha) p_{t-1} M,   M = D^-1 A  (Sec. 3),
 * for k independent teleport vectors p_0 (columns of the n x k p0).
 * A row u with d_u = 0 has no row in D^-1 A; its mass is spread over a
 * fixed distribution g: p_{t-1} M is read as (p_{t-1} D^-1) A + delta g with
 * delta = sum_{d_u = 0} p_{t-1,u}, which keeps sum p_t = 1. g = p_0 when
 * dangling == 0 (default), g = 1/n when dangling == 1.
 * Start: p_init if given, else p_0 (the uniform start for p_0 = 1/n).
 * Stops after the first update whose L1 change ||p_t - p_{t-1}||_1 < tol in
 * every column, or after max_iter updates. No renormalisation is applied.
 * Returns the number of updates; resid[c] = last L1 change of column c.
 */
int32_t oracle_pagerank(int64_t n, const int64_t* rp, const int32_t* ci, double alpha,
                        const double* p0, const double* p_init, int32_t k, double tol,
                        int32_t max_iter, int32_t dangling, double* p, double* resid) {
    double* x = (double*)malloc(sizeof(double) * (size_t)(n * k > 0 ? n * k : 1));
    double* y = (double*)malloc(sizeof(double) * (size_t)(n * k > 0 ? n * k : 1));
    double* delta = (double*)malloc(sizeof(double) * (size_t)k);
    memcpy(p, p_init ? p_init : p0, sizeof(double) * (size_t)(n * k));
    int32_t it = 0;
    for (int32_t c = 0; c < k; c++) resid[c] = INFINITY;
    while (it < max_iter) {
        for (int32_t c = 0; c < k; c++) delta[c] = 0.0;
        for (int64_t u = 0; u < n; u++) {
            int64_t d = rp[u + 1] - rp[u];
            for (int32_t c = 0; c < k; c++) {
                if (d == 0) {
                    x[u * k + c] = 0.0;
                    delta[c] += p[u * k + c];
                } else {
                    x[u * k + c] = p[u * k + c] / (double)d;
                }
            }
        }
        oracle_csr_xA(n, rp, ci, x, k, y);
        for (int32_t c = 0; c < k; c++) resid[c] = 0.0;
        for (int64_t v = 0; v < n; v++) {
            for (int32_t c = 0; c < k; c++) {
                double g = dangling == 1 ? 1.0 / (double)n : p0[v * k + c];
                double pn = alpha * p0[v * k + c] + (1.0 - alpha) * (y[v * k + c] + delta[c] * g);
                resid[c] += fabs(pn - p[v * k + c]);
                p[v * k + c] = pn;
            }
        }
        it++;
        int done = 1;
        for (int32_t c = 0; c < k; c++)
            if (!(resid[c] < tol)) done = 0;
        if (done) break;
    }
    free(x);
    free(y);
    free(delta);
    return it;
}

/*
 * Seeded synthetic graph generator: a copying model for web-like and
 * social-like adjacency matrices.
 *
 * This file produces INPUTS only. It holds none of the compressed-product
 * arithmetic: both the CUDA library and the CPU oracle consume the CSR it
 * writes. It stands in for the LAW web and social crawls of the paper's
 * Table 1 (which are not available here) with their shape: rows of nearby
 * nodes copy each other's successor lists (the copy property of Sec. 4),
 * successors are local ids and runs of consecutive ids.
 *
 * Model (one row at a time, row i in increasing order):
 *   - with probability p_copy the row is a copy row: it picks a prototype u
 *     uniformly among the previous `window` rows, keeps each successor of u
 *     independently with probability `fidelity`, then adds Geom(extra_mean)
 *     new slots;
 *   - otherwise it is a fresh row: its degree d is drawn (geometric with
 *     mean fresh_mean, or a power law with exponent alpha on [dmin, dmax])
 *     and slots are added until it holds d successors;
 *   - a slot is a run (with probability q_run) of U{run_min..run_max}
 *     consecutive ids starting at a local position, or one id; a local
 *     position is i +- Geom(gap_mean); with random_ids the single ids are
 *     uniform over [0, n) instead.
 *   - rows are sorted and de-duplicated.
 *
 * Random numbers come from a counter-based splitmix64 stream per row
 * (state = mix(seed, row)), so the output is a pure function of the
 * parameters. No libm call is used: geometric and power-law draws use
 * tables built with IEEE +,-,*,/ only, so x86 and Arm hosts produce the
 * same graph bit for bit.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int64_t n;
    uint64_t seed;
    double p_copy;
    double fidelity;
    double extra_mean;
    double fresh_mean;
    int32_t powerlaw;
    double alpha;
    int64_t dmin;
    int64_t dmax;
    double q_run;
    int32_t run_min;
    int32_t run_max;
    double gap_mean;
    int32_t random_ids;
    int32_t window;
} synth_params;

static inline uint64_t sm64_next(uint64_t* s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* U[0,1) with 53 random bits. */
static inline double unif(uint64_t* s) {
    return (double)(sm64_next(s) >> 11) * (1.0 / 9007199254740992.0);
}

/* Table of survival thresholds for a geometric law on {0,1,2,...} with the
 * given mean: T[k] = q^k with q = mean/(mean+1). A draw is the number of
 * k >= 1 with T[k] > U. */
typedef struct {
    double* t;
    int64_t len;
} geom_table;

static int geom_init(geom_table* g, double mean) {
    g->t = NULL;
    g->len = 0;
    if (mean <= 0.0) return 0;
    double q = mean / (mean + 1.0);
    int64_t cap = 1024;
    g->t = (double*)malloc(sizeof(double) * cap);
    if (!g->t) return -1;
    double v = 1.0;
    while (v > 1e-18) {
        if (g->len == cap) {
            cap *= 2;
            double* nt = (double*)realloc(g->t, sizeof(double) * cap);
            if (!nt) return -1;
            g->t = nt;
        }
        g->t[g->len++] = v;
        v *= q;
    }
    return 0;
}

static int64_t geom_draw(const geom_table* g, uint64_t* s) {
    if (g->len == 0) return 0;
    double u = unif(s);
    /* count k >= 1 with t[k] > u; t is decreasing */
    int64_t lo = 1, hi = g->len; /* answer in [0, len-1] */
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (g->t[mid] > u) lo = mid + 1; else hi = mid;
    }
    return lo - 1;
}

/* Natural log and exp by series, IEEE basic ops only (for table building). */
static double my_log(double x) {
    /* x > 0: x = m * 2^e with m in [1,2) */
    int e = 0;
    while (x >= 2.0) { x *= 0.5; e++; }
    while (x < 1.0) { x *= 2.0; e--; }
    double t = (x - 1.0) / (x + 1.0), t2 = t * t, term = t, sum = 0.0;
    for (int k = 1; k < 80; k += 2) { sum += term / k; term *= t2; }
    return 2.0 * sum + e * 0.69314718055994530942;
}

static double my_exp(double x) {
    /* exp(x) = 2^j * exp(r), |r| <= ln2/2 */
    const double ln2 = 0.69314718055994530942;
    double jd = x / ln2;
    int64_t j = (int64_t)(jd < 0 ? jd - 0.5 : jd + 0.5);
    double r = x - (double)j * ln2, term = 1.0, sum = 1.0;
    for (int k = 1; k < 30; k++) { term *= r / k; sum += term; }
    while (j > 0) { sum *= 2.0; j--; }
    while (j < 0) { sum *= 0.5; j++; }
    return sum;
}

/* Power law P(D >= d) = (d/dmin)^-(alpha-1) on [dmin, dmax]: thresholds. */
typedef struct {
    double* t;
    int64_t dmin, dmax;
} pl_table;

static int pl_init(pl_table* p, double alpha, int64_t dmin, int64_t dmax) {
    p->dmin = dmin;
    p->dmax = dmax;
    int64_t len = dmax - dmin + 2;
    p->t = (double*)malloc(sizeof(double) * len);
    if (!p->t) return -1;
    double tail = my_exp(-(alpha - 1.0) * my_log((double)(dmax + 1) / (double)dmin));
    for (int64_t k = 0; k < len; k++) {
        double d = (double)(dmin + k);
        double s = my_exp(-(alpha - 1.0) * my_log(d / (double)dmin));
        /* truncated and renormalised survival function */
        p->t[k] = (s - tail) / (1.0 - tail);
    }
    return 0;
}

static int64_t pl_draw(const pl_table* p, uint64_t* s) {
    double u = unif(s);
    /* largest k with t[k] > u  ->  degree dmin + k */
    int64_t lo = 0, hi = p->dmax - p->dmin; /* t[0] = 1 > u always */
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (p->t[mid] > u) lo = mid; else hi = mid - 1;
    }
    return p->dmin + lo;
}

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

static void sort_i32(int32_t* a, int64_t len) {
    if (len < 24) {
        for (int64_t i = 1; i < len; i++) {
            int32_t v = a[i];
            int64_t j = i - 1;
            while (j >= 0 && a[j] > v) { a[j + 1] = a[j]; j--; }
            a[j + 1] = v;
        }
    } else {
        qsort(a, (size_t)len, sizeof(int32_t), cmp_i32);
    }
}

typedef struct {
    int32_t* v;
    int64_t len, cap;
} ivec;

static int iv_push(ivec* a, int32_t x) {
    if (a->len == a->cap) {
        int64_t nc = a->cap ? a->cap * 2 : 1024;
        int32_t* nv = (int32_t*)realloc(a->v, sizeof(int32_t) * nc);
        if (!nv) return -1;
        a->v = nv;
        a->cap = nc;
    }
    a->v[a->len++] = x;
    return 0;
}

static int64_t local_pos(int64_t i, int64_t n, const geom_table* gap, uint64_t* s) {
    int64_t g = geom_draw(gap, s) + 1;
    int64_t j = (sm64_next(s) & 1) ? i + g : i - g;
    if (j < 0) j = -j;            /* reflect at the borders */
    if (j >= n) j = 2 * (n - 1) - j;
    if (j < 0) j = 0;
    return j;
}

/* Adds one slot to `row`; returns the number of ids appended or -1. */
static int64_t add_slot(ivec* row, int64_t i, const synth_params* P,
                        const geom_table* gap, uint64_t* s, int64_t room) {
    int64_t n = P->n;
    if (room <= 0) return 0;
    if (P->q_run > 0.0 && unif(s) < P->q_run) {
        int64_t span = P->run_max - P->run_min + 1;
        int64_t len = P->run_min + (int64_t)(sm64_next(s) % (uint64_t)span);
        if (len > room) len = room;
        int64_t st = local_pos(i, n, gap, s);
        if (st + len > n) st = n - len;
        if (st < 0) { st = 0; if (len > n) len = n; }
        for (int64_t t = 0; t < len; t++)
            if (iv_push(row, (int32_t)(st + t))) return -1;
        return len;
    }
    int64_t j;
    if (P->random_ids) j = (int64_t)(sm64_next(s) % (uint64_t)n);
    else j = local_pos(i, n, gap, s);
    if (iv_push(row, (int32_t)j)) return -1;
    return 1;
}

/* Generates the graph. On success *row_ptr (n+1) and *col (m) are malloc'd
 * and owned by the caller (free with synth_free). Returns 0, or -1 on bad
 * parameters or allocation failure. */
int synth_copying_model(const synth_params* P, int64_t** row_ptr_out, int32_t** col_out,
                        int64_t* m_out) {
    if (!P || !row_ptr_out || !col_out || !m_out) return -1;
    int64_t n = P->n;
    if (n <= 0 || n > 2147483647LL || P->window < 1) return -1;
    if (P->run_min < 1 || P->run_max < P->run_min) return -1;
    if (P->powerlaw && (P->dmin < 1 || P->dmax < P->dmin || P->alpha <= 1.0)) return -1;

    geom_table gap = {0}, extra = {0}, fresh = {0};
    pl_table pl = {0};
    int64_t* rp = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
    ivec col = {0}, row = {0};
    int rc = -1;
    if (!rp) goto done;
    if (geom_init(&gap, P->gap_mean) || geom_init(&extra, P->extra_mean) ||
        geom_init(&fresh, P->fresh_mean))
        goto done;
    if (P->powerlaw && pl_init(&pl, P->alpha, P->dmin, P->dmax)) goto done;

    rp[0] = 0;
    for (int64_t i = 0; i < n; i++) {
        uint64_t s = P->seed * 0xD1B54A32D192ED03ULL ^ ((uint64_t)i * 0x9E3779B97F4A7C15ULL);
        sm64_next(&s);
        row.len = 0;
        int64_t cap = n;  /* a row cannot hold more than n distinct ids */
        if (i > 0 && unif(&s) < P->p_copy) {
            int64_t w = i < P->window ? i : P->window;
            int64_t u = i - 1 - (int64_t)(sm64_next(&s) % (uint64_t)w);
            for (int64_t e = rp[u]; e < rp[u + 1]; e++)
                if (unif(&s) < P->fidelity && iv_push(&row, col.v[e])) goto done;
            int64_t ex = geom_draw(&extra, &s);
            for (int64_t t = 0; t < ex; t++)
                if (add_slot(&row, i, P, &gap, &s, cap - row.len) < 0) goto done;
        } else {
            int64_t d = P->powerlaw ? pl_draw(&pl, &s) : geom_draw(&fresh, &s) + 1;
            if (d > cap) d = cap;
            int64_t guard = 0;
            while (row.len < d && guard < 64 * d + 64) {
                if (add_slot(&row, i, P, &gap, &s, d - row.len) < 0) goto done;
                guard++;
            }
        }
        sort_i32(row.v, row.len);
        int64_t k = 0;
        for (int64_t t = 0; t < row.len; t++)
            if (k == 0 || row.v[t] != row.v[k - 1]) row.v[k++] = row.v[t];
        for (int64_t t = 0; t < k; t++)
            if (iv_push(&col, row.v[t])) goto done;
        rp[i + 1] = col.len;
    }
    *row_ptr_out = rp;
    *col_out = col.v ? col.v : (int32_t*)malloc(sizeof(int32_t));
    *m_out = col.len;
    rp = NULL;
    col.v = NULL;
    rc = 0;
done:
    free(rp);
    free(col.v);
    free(row.v);
    free(gap.t);
    free(extra.t);
    free(fresh.t);
    free(pl.t);
    return rc;
}

void synth_free(void* p) { free(p); }

/* x[i] = U[0,1) with 53 random bits from the stream of (seed, i): the
 * right-hand sides of the products (FP64; callers round to FP32). */
void synth_uniform(int64_t count, uint64_t seed, double* out) {
    for (int64_t i = 0; i < count; i++) {
        uint64_t s = seed * 0xD1B54A32D192ED03ULL ^ ((uint64_t)i * 0x9E3779B97F4A7C15ULL);
        sm64_next(&s);
        out[i] = unif(&s);
    }
}

/* Draws `count` distinct-by-stream node ids uniformly in [0, n). */
void synth_nodes(int64_t count, int64_t n, uint64_t seed, int64_t* out) {
    for (int64_t i = 0; i < count; i++) {
        uint64_t s = (seed + 0x5851F42D4C957F2DULL) * 0xD1B54A32D192ED03ULL ^
                     ((uint64_t)i * 0x9E3779B97F4A7C15ULL);
        sm64_next(&s);
        out[i] = (int64_t)(sm64_next(&s) % (uint64_t)n);
    }
}

// Host encoder of the BV-delta representation: reference choice (Sec. 4
// window, Sec. 5 keep-raw rule), split of each difference row into dropped
// ids, intervals and residual ids, and a gamma/delta-coded bitstream with its
// decoder (used for the bits/edge statistic and the round trip).
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>

#include "bvg_internal.h"

namespace bvg {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

// Allocation-failure injection for tests: the checkpoint reached when the
// counter is 0 fails once (the counter then stays at -1, disabled).
static std::atomic<int64_t> g_fail_alloc_after{-1};
bool inject_alloc_failure() {
    int64_t v = g_fail_alloc_after.load();
    while (v >= 0)
        if (g_fail_alloc_after.compare_exchange_weak(v, v - 1)) return v == 0;
    return false;
}

int fail(int status, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return status;
}

const char* last_error() { return g_last_error.c_str(); }

namespace {

// Cost of writing row vi against reference vr (sorted, duplicate-free):
// one word per dropped id, per residual id, two per interval (maximal run of
// >= lmin consecutive added ids). sym = |vi xor vr| = nnz of the difference row.
struct Cost {
    int64_t cost, sym;
};

Cost diff_cost(const int32_t* vi, int64_t ni, const int32_t* vr, int64_t nr, int lmin) {
    int64_t a = 0, b = 0, dropped = 0, added = 0, residual = 0, intervals = 0;
    int64_t run_len = 0;
    int32_t run_end = 0;  // last id of the current run
    auto close_run = [&]() {
        if (run_len >= lmin) intervals++;
        else residual += run_len;
        run_len = 0;
    };
    auto add = [&](int32_t j) {
        added++;
        if (run_len > 0 && j == run_end + 1) {
            run_len++;
        } else {
            if (run_len > 0) close_run();
            run_len = 1;
        }
        run_end = j;
    };
    while (a < ni || b < nr) {
        if (b >= nr || (a < ni && vi[a] < vr[b])) add(vi[a++]);
        else if (a >= ni || vr[b] < vi[a]) { dropped++; b++; }
        else { a++; b++; }
    }
    if (run_len > 0) close_run();
    return {dropped + residual + 2 * intervals, dropped + added};
}

template <class F>
void parallel_for(int64_t n, int threads, F&& f) {
    if (threads <= 1 || n < 4096) {
        f(0, n);
        return;
    }
    std::vector<std::thread> pool;
    std::atomic<int64_t> next{0};
    const int64_t chunk = std::max<int64_t>(1024, n / (threads * 8));
    for (int t = 0; t < threads; t++) {
        pool.emplace_back([&]() {
            for (;;) {
                int64_t s = next.fetch_add(chunk);
                if (s >= n) break;
                f(s, std::min(n, s + chunk));
            }
        });
    }
    for (auto& th : pool) th.join();
}

// ---- bit I/O (MSB first within 64-bit words) ---------------------------
struct BitWriter {
    std::vector<uint64_t>& w;
    int64_t nbits = 0;
    explicit BitWriter(std::vector<uint64_t>& v) : w(v) {}
    void put(uint64_t value, int len) {  // len <= 64, low `len` bits of value
        for (int i = len - 1; i >= 0; i--) {
            if ((nbits & 63) == 0) w.push_back(0);
            if ((value >> i) & 1) w.back() |= (uint64_t)1 << (63 - (nbits & 63));
            nbits++;
        }
    }
    void zeros(int len) {
        for (int i = 0; i < len; i++) {
            if ((nbits & 63) == 0) w.push_back(0);
            nbits++;
        }
    }
    static int bitlen(uint64_t x) { return 64 - __builtin_clzll(x); }
    void gamma(uint64_t x) {  // x >= 1
        int L = bitlen(x);
        zeros(L - 1);
        put(x, L);
    }
    void delta(uint64_t x) {  // x >= 1
        int L = bitlen(x);
        gamma((uint64_t)L);
        put(x, L - 1);
    }
};

struct BitReader {
    const uint64_t* w;
    int64_t nbits, pos = 0;
    bool bad = false;
    BitReader(const uint64_t* words, int64_t n) : w(words), nbits(n) {}
    int bit() {
        if (pos >= nbits) { bad = true; return 0; }
        int b = (int)((w[pos >> 6] >> (63 - (pos & 63))) & 1);
        pos++;
        return b;
    }
    uint64_t get(int len) {
        uint64_t v = 0;
        for (int i = 0; i < len; i++) v = (v << 1) | (uint64_t)bit();
        return v;
    }
    uint64_t gamma() {
        int z = 0;
        while (!bad && bit() == 0) {
            if (++z > 63) { bad = true; return 1; }
        }
        if (bad) return 1;
        return ((uint64_t)1 << z) | get(z);
    }
    uint64_t delta() {
        uint64_t L = gamma();
        if (bad || L < 1 || L > 64) { bad = true; return 1; }
        return ((uint64_t)1 << (L - 1)) | get((int)L - 1);
    }
};

inline uint64_t fold(int64_t v) { return v >= 0 ? (uint64_t)(2 * v) : (uint64_t)(-2 * v - 1); }
inline int64_t unfold(uint64_t u) { return (u & 1) ? -(int64_t)((u + 1) / 2) : (int64_t)(u / 2); }

}  // namespace

// Splits row i against its reference into dropped ids, intervals, residual
// ids (appending to the given vectors).
static void split_row(const int32_t* vi, int64_t ni, const int32_t* vr, int64_t nr, int lmin, int32_t* drop,
                      int64_t* nd, int32_t* res, int64_t* nres, int32_t* ivs, int32_t* ivl, int64_t* niv) {
    int64_t a = 0, b = 0;
    int64_t run_len = 0;
    int32_t run_start = 0;
    *nd = *nres = *niv = 0;
    auto close_run = [&]() {
        if (run_len >= lmin) {
            ivs[*niv] = run_start;
            ivl[*niv] = (int32_t)run_len;
            (*niv)++;
        } else {
            for (int64_t t = 0; t < run_len; t++) res[(*nres)++] = run_start + (int32_t)t;
        }
        run_len = 0;
    };
    auto add = [&](int32_t j) {
        if (run_len > 0 && j == run_start + run_len) {
            run_len++;
        } else {
            if (run_len > 0) close_run();
            run_start = j;
            run_len = 1;
        }
    };
    while (a < ni || b < nr) {
        if (b >= nr || (a < ni && vi[a] < vr[b])) add(vi[a++]);
        else if (a >= ni || vr[b] < vi[a]) drop[(*nd)++] = vr[b++];
        else { a++; b++; }
    }
    if (run_len > 0) close_run();
}

}  // namespace bvg

using namespace bvg;

extern "C" const char* bvg_last_error(void) { return bvg::last_error(); }

extern "C" int bvg_debug_fail_alloc(int64_t after) {
    bvg::g_fail_alloc_after.store(after < 0 ? -1 : after);
    return BVG_OK;
}

// The encoder for an n x ncols block of rows (ids in [0, ncols)): references
// are chosen among the block's own rows. bvg_encode is the square case.
int bvg::encode_rows(int64_t n, int64_t ncols, const int64_t* row_ptr, const int32_t* col_idx,
                     const bvg_encode_params* params, bvg_host_graph** out) {
    if (!out) return fail(BVG_ERR_INVALID_ARG, "bvg_encode: out is NULL");
    *out = nullptr;
    if (n < 0 || !row_ptr || (n > 0 && row_ptr[n] > 0 && !col_idx))
        return fail(BVG_ERR_INVALID_ARG, "bvg_encode: bad n or NULL arrays");
    if (n >= kMaxN || ncols >= kMaxN || ncols < 0)
        return fail(BVG_ERR_UNSUPPORTED, "bvg_encode: n = %lld exceeds 2^30 - 1", (long long)std::max(n, ncols));
    int W = params && params->window ? params->window : 7;
    int R = params && params->max_chain ? params->max_chain : 3;
    int L = params && params->min_interval ? params->min_interval : 4;
    int threads = params && params->threads > 0 ? params->threads : (int)std::thread::hardware_concurrency();
    if (threads < 1) threads = 1;
    if (W < 1 || W > kMaxWindow || R < 1 || R > kMaxChain || W * R > kMaxSpan || L < 2)
        return fail(BVG_ERR_UNSUPPORTED, "bvg_encode: window %d / max_chain %d / min_interval %d unsupported "
                                         "(window 1..31, max_chain 1..3, window * max_chain <= 32, "
                                         "min_interval >= 2)", W, R, L);
    // ---- validate CSR
    if (row_ptr[0] != 0) return fail(BVG_ERR_BAD_GRAPH, "bvg_encode: row_ptr[0] != 0");
    for (int64_t i = 0; i < n; i++) {
        if (row_ptr[i + 1] < row_ptr[i]) return fail(BVG_ERR_BAD_GRAPH, "bvg_encode: row_ptr decreases at row %lld", (long long)i);
        if (row_ptr[i + 1] - row_ptr[i] > ncols)
            return fail(BVG_ERR_BAD_GRAPH, "bvg_encode: row %lld longer than n", (long long)i);
    }
    const int64_t m = n > 0 ? row_ptr[n] : 0;
    std::atomic<int64_t> bad_row{-1};
    parallel_for(n, threads, [&](int64_t s, int64_t e) {
        for (int64_t i = s; i < e; i++) {
            for (int64_t t = row_ptr[i]; t < row_ptr[i + 1]; t++) {
                int32_t j = col_idx[t];
                if (j < 0 || j >= ncols || (t > row_ptr[i] && col_idx[t - 1] >= j)) {
                    int64_t expect = -1;
                    bad_row.compare_exchange_strong(expect, i);
                    return;
                }
            }
        }
    });
    if (bad_row.load() >= 0)
        return fail(BVG_ERR_BAD_GRAPH, "bvg_encode: row %lld has an unsorted, duplicate or out-of-range id",
                    (long long)bad_row.load());

    bvg_host_graph* g = new (std::nothrow) bvg_host_graph();
    if (!g) return fail(BVG_ERR_OOM, "bvg_encode: host allocation failed");
    try {
        if (inject_alloc_failure()) throw std::bad_alloc();
        g->n = n;
        g->m = m;
        g->window = W;
        g->max_chain = R;
        g->min_interval = L;
        g->ref.assign(n, -1);
        g->depth.assign(n, 0);
        g->outdeg.resize(n);
        for (int64_t i = 0; i < n; i++) g->outdeg[i] = (uint32_t)(row_ptr[i + 1] - row_ptr[i]);

        // ---- reference choice: costs in parallel, selection in row order
        const int64_t B = 1 << 20;
        std::vector<int64_t> cost((size_t)std::min<int64_t>(B, std::max<int64_t>(n, 1)) * (W + 1));
        std::vector<int64_t> sym((size_t)std::min<int64_t>(B, std::max<int64_t>(n, 1)) * (W + 1));
        for (int64_t b0 = 0; b0 < n; b0 += B) {
            int64_t b1 = std::min(n, b0 + B);
            parallel_for(b1 - b0, threads, [&](int64_t s, int64_t e) {
                for (int64_t ii = s; ii < e; ii++) {
                    int64_t i = b0 + ii;
                    const int32_t* vi = col_idx + row_ptr[i];
                    int64_t ni = row_ptr[i + 1] - row_ptr[i];
                    Cost raw = diff_cost(vi, ni, nullptr, 0, L);
                    cost[ii * (W + 1)] = raw.cost;
                    sym[ii * (W + 1)] = raw.sym;
                    for (int w = 1; w <= W; w++) {
                        int64_t r = i - w;
                        if (r < 0) break;
                        Cost c = diff_cost(vi, ni, col_idx + row_ptr[r], row_ptr[r + 1] - row_ptr[r], L);
                        cost[ii * (W + 1) + w] = c.cost;
                        sym[ii * (W + 1) + w] = c.sym;
                    }
                }
            });
            for (int64_t i = b0; i < b1; i++) {
                int64_t ii = i - b0;
                int64_t best = -1, best_cost = 0, best_sym = 0;
                for (int w = 1; w <= W && i - w >= 0; w++) {
                    if (g->depth[i - w] >= R) continue;
                    int64_t c = cost[ii * (W + 1) + w];
                    if (best < 0 || c < best_cost) {
                        best = i - w;
                        best_cost = c;
                        best_sym = sym[ii * (W + 1) + w];
                    }
                }
                int64_t deg = row_ptr[i + 1] - row_ptr[i];
                if (best >= 0 && best_cost < cost[ii * (W + 1)] && best_sym < deg) {
                    g->ref[i] = (int32_t)best;
                    g->depth[i] = (uint8_t)(g->depth[best] + 1);
                }
            }
        }

        // ---- split rows: sizes, offsets, fill
        std::vector<int64_t> nd(n), nr(n), ni(n);
        parallel_for(n, threads, [&](int64_t s, int64_t e) {
            std::vector<int32_t> d, r, a, b;
            for (int64_t i = s; i < e; i++) {
                const int32_t* vi = col_idx + row_ptr[i];
                int64_t li = row_ptr[i + 1] - row_ptr[i];
                int64_t rr = g->ref[i];
                const int32_t* vr = rr >= 0 ? col_idx + row_ptr[rr] : nullptr;
                int64_t lr = rr >= 0 ? row_ptr[rr + 1] - row_ptr[rr] : 0;
                d.resize(lr + 1);
                r.resize(li + 1);
                a.resize(li + 1);
                b.resize(li + 1);
                split_row(vi, li, vr, lr, L, d.data(), &nd[i], r.data(), &nr[i], a.data(), b.data(), &ni[i]);
            }
        });
        g->drop_ptr.resize(n + 1);
        g->res_ptr.resize(n + 1);
        g->iv_ptr.resize(n + 1);
        g->drop_ptr[0] = g->res_ptr[0] = g->iv_ptr[0] = 0;
        for (int64_t i = 0; i < n; i++) {
            g->drop_ptr[i + 1] = g->drop_ptr[i] + nd[i];
            g->res_ptr[i + 1] = g->res_ptr[i] + nr[i];
            g->iv_ptr[i + 1] = g->iv_ptr[i] + ni[i];
        }
        g->drop.resize(g->drop_ptr[n]);
        g->res.resize(g->res_ptr[n]);
        g->iv_s.resize(g->iv_ptr[n]);
        g->iv_len.resize(g->iv_ptr[n]);
        parallel_for(n, threads, [&](int64_t s, int64_t e) {
            for (int64_t i = s; i < e; i++) {
                const int32_t* vi = col_idx + row_ptr[i];
                int64_t li = row_ptr[i + 1] - row_ptr[i];
                int64_t rr = g->ref[i];
                const int32_t* vr = rr >= 0 ? col_idx + row_ptr[rr] : nullptr;
                int64_t lr = rr >= 0 ? row_ptr[rr + 1] - row_ptr[rr] : 0;
                int64_t a, b, c;
                split_row(vi, li, vr, lr, L, g->drop.data() + g->drop_ptr[i], &a, g->res.data() + g->res_ptr[i], &b,
                          g->iv_s.data() + g->iv_ptr[i], g->iv_len.data() + g->iv_ptr[i], &c);
            }
        });

        // ---- bitstream
        BitWriter bw(g->bits);
        for (int64_t i = 0; i < n; i++) {
            int64_t rr = g->ref[i];
            bw.gamma(rr >= 0 ? (uint64_t)(i - rr + 1) : 1);
            if (rr >= 0) {
                // copy blocks over v_r: alternating kept / dropped runs, kept first
                const int32_t* vr = col_idx + row_ptr[rr];
                int64_t lr = row_ptr[rr + 1] - row_ptr[rr];
                const int32_t* dp = g->drop.data() + g->drop_ptr[i];
                int64_t ndr = g->drop_ptr[i + 1] - g->drop_ptr[i], t = 0;
                std::vector<int64_t> blocks;
                int64_t cur = 0;
                bool kept = true;
                for (int64_t e = 0; e < lr; e++) {
                    bool is_drop = t < ndr && dp[t] == vr[e];
                    if (is_drop) t++;
                    if (is_drop == kept) {  // state flips
                        blocks.push_back(cur);
                        cur = 0;
                        kept = !kept;
                    }
                    cur++;
                }
                if (lr > 0) blocks.push_back(cur);
                bw.gamma(blocks.size() + 1);
                for (size_t b = 0; b + 1 < blocks.size(); b++) bw.gamma(b == 0 ? blocks[b] + 1 : blocks[b]);
            }
            int64_t niv = g->iv_ptr[i + 1] - g->iv_ptr[i];
            bw.gamma(niv + 1);
            int64_t prev_end = 0;
            for (int64_t t = 0; t < niv; t++) {
                int64_t s0 = g->iv_s[g->iv_ptr[i] + t], len = g->iv_len[g->iv_ptr[i] + t];
                if (t == 0) bw.delta(fold(s0 - i) + 1);
                else bw.delta((uint64_t)(s0 - prev_end));
                bw.gamma((uint64_t)(len - L + 1));
                prev_end = s0 + len;
            }
            int64_t nres = g->res_ptr[i + 1] - g->res_ptr[i];
            bw.gamma(nres + 1);
            int64_t prev = 0;
            for (int64_t t = 0; t < nres; t++) {
                int64_t j = g->res[g->res_ptr[i] + t];
                if (t == 0) bw.delta(fold(j - i) + 1);
                else bw.delta((uint64_t)(j - prev));
                prev = j;
            }
        }
        g->nbits = bw.nbits;

        // ---- stats
        bvg_graph_stats& st = g->stats;
        memset(&st, 0, sizeof(st));
        st.n = n;
        st.m = m;
        st.dropped = g->drop_ptr[n];
        st.residual = g->res_ptr[n];
        st.intervals = g->iv_ptr[n];
        for (int64_t t = 0; t < st.intervals; t++) st.interval_members += g->iv_len[t];
        st.added = st.residual + st.interval_members;
        st.nnz_diff = st.dropped + st.added;
        st.words = st.dropped + st.residual + 2 * st.intervals;
        for (int64_t i = 0; i < n; i++) {
            st.rows_with_ref += g->ref[i] >= 0;
            st.depth_hist[g->depth[i]]++;
        }
        st.bitstream_bits = g->nbits;
        st.bits_per_edge = m > 0 ? (double)g->nbits / (double)m : 0.0;
        int64_t ends = 0;
        for (int64_t t = 0; t < st.intervals; t++) ends += (int64_t)g->iv_s[t] + g->iv_len[t] < ncols;
        int64_t tiles = (n + kCarryTile - 1) / kCarryTile;
        int64_t carry = 0;
        for (int64_t t = 0; t < st.intervals; t++) {
            int64_t s0 = g->iv_s[t], e0 = std::min<int64_t>(s0 + g->iv_len[t], tiles * kCarryTile - 1);
            carry += e0 / kCarryTile - s0 / kCarryTile;
        }
        st.device_bytes = n * 1 + 4 * (n + 1) + 4 * st.words        // row-major
                          + 4 * (n + 1) + 4 * (st.dropped + st.residual + st.intervals + ends)  // column-major
                          + 4 * (tiles + 1) + 4 * carry + 4 * n;    // carry lists, 1/outdeg
    } catch (const std::bad_alloc&) {
        delete g;
        return fail(BVG_ERR_OOM, "bvg_encode: host allocation failed");
    }
    *out = g;
    return BVG_OK;
}

extern "C" int bvg_encode(int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
                          const bvg_encode_params* params, bvg_host_graph** out) {
    return encode_rows(n, n, row_ptr, col_idx, params, out);
}

// Decodes a bitstream of n rows and m edges written with window W and minimum
// interval length L into caller buffers row_ptr[n + 1], col_idx[m]. Every
// count, offset and id read from the stream is checked against n, m, W and
// the rows already decoded before it is used, so a damaged or truncated
// stream gives BVG_ERR_CORRUPT and never an access outside the buffers.
static int decode_stream(int64_t n, int64_t m, int W, int L, const uint64_t* bits, int64_t nbits,
                         int64_t* row_ptr, int32_t* col_idx) {
    BitReader br(bits, nbits);
    row_ptr[0] = 0;
    int64_t pos = 0;
    std::vector<int32_t> kept, ivs, res;
    for (int64_t i = 0; i < n; i++) {
        kept.clear();
        ivs.clear();
        res.clear();
        uint64_t off = br.gamma() - 1;
        if (br.bad || (int64_t)off > i || off > (uint64_t)W)
            return fail(BVG_ERR_CORRUPT, "bvg_decode: bad reference at row %lld", (long long)i);
        if (off > 0) {
            int64_t rr = i - (int64_t)off;
            int64_t lr = row_ptr[rr + 1] - row_ptr[rr];
            uint64_t nb = br.gamma() - 1;
            if (br.bad || (int64_t)nb > lr + 1 || (lr > 0) != (nb > 0))
                return fail(BVG_ERR_CORRUPT, "bvg_decode: bad copy-block count at row %lld", (long long)i);
            int64_t e = 0;
            bool keep = true;
            for (uint64_t b = 0; b < nb; b++) {
                int64_t len;
                if (b + 1 < nb) {
                    uint64_t v = br.gamma();
                    len = b == 0 ? (int64_t)v - 1 : (int64_t)v;
                } else {
                    len = lr - e;
                }
                if (br.bad || len < 0 || e + len > lr || (b > 0 && len < 1))
                    return fail(BVG_ERR_CORRUPT, "bvg_decode: bad copy block at row %lld", (long long)i);
                if (keep && pos + (int64_t)kept.size() + len > m)
                    return fail(BVG_ERR_CORRUPT, "bvg_decode: more edges than m at row %lld", (long long)i);
                if (keep)
                    for (int64_t t = 0; t < len; t++) kept.push_back(col_idx[row_ptr[rr] + e + t]);
                e += len;
                keep = !keep;
            }
        }
        uint64_t niv = br.gamma() - 1;
        if (br.bad || (int64_t)niv > n) return fail(BVG_ERR_CORRUPT, "bvg_decode: bad interval count at row %lld", (long long)i);
        int64_t prev_end = 0;
        for (uint64_t t = 0; t < niv; t++) {
            int64_t s0 = t == 0 ? i + unfold(br.delta() - 1) : prev_end + (int64_t)br.delta();
            int64_t len = (int64_t)br.gamma() + L - 1;
            if (br.bad || s0 < 0 || len < L || s0 + len > n)
                return fail(BVG_ERR_CORRUPT, "bvg_decode: bad interval at row %lld", (long long)i);
            if (pos + (int64_t)(kept.size() + ivs.size()) + len > m)
                return fail(BVG_ERR_CORRUPT, "bvg_decode: more edges than m at row %lld", (long long)i);
            for (int64_t q = 0; q < len; q++) ivs.push_back((int32_t)(s0 + q));
            prev_end = s0 + len;
        }
        uint64_t nres = br.gamma() - 1;
        if (br.bad || (int64_t)nres > n) return fail(BVG_ERR_CORRUPT, "bvg_decode: bad residual count at row %lld", (long long)i);
        int64_t prev = 0;
        for (uint64_t t = 0; t < nres; t++) {
            int64_t j = t == 0 ? i + unfold(br.delta() - 1) : prev + (int64_t)br.delta();
            if (br.bad || j < 0 || j >= n) return fail(BVG_ERR_CORRUPT, "bvg_decode: bad residual at row %lld", (long long)i);
            if (pos + (int64_t)(kept.size() + ivs.size() + res.size()) + 1 > m)
                return fail(BVG_ERR_CORRUPT, "bvg_decode: more edges than m at row %lld", (long long)i);
            res.push_back((int32_t)j);
            prev = j;
        }
        // merge the three sorted lists
        size_t total = kept.size() + ivs.size() + res.size();
        if (pos + (int64_t)total > m) return fail(BVG_ERR_CORRUPT, "bvg_decode: more edges than m at row %lld", (long long)i);
        int32_t* outp = col_idx + pos;
        std::vector<int32_t> tmp(kept.size() + ivs.size());
        std::merge(kept.begin(), kept.end(), ivs.begin(), ivs.end(), tmp.begin());
        std::merge(tmp.begin(), tmp.end(), res.begin(), res.end(), outp);
        for (size_t t = 1; t < total; t++)
            if (outp[t - 1] >= outp[t]) return fail(BVG_ERR_CORRUPT, "bvg_decode: overlapping entries at row %lld", (long long)i);
        pos += (int64_t)total;
        row_ptr[i + 1] = pos;
    }
    if (pos != m || br.pos != nbits) return fail(BVG_ERR_CORRUPT, "bvg_decode: stream length mismatch");
    return BVG_OK;
}

extern "C" int bvg_decode(const bvg_host_graph* g, int64_t* row_ptr, int32_t* col_idx) {
    if (!g || !row_ptr || (g->m > 0 && !col_idx)) return fail(BVG_ERR_INVALID_ARG, "bvg_decode: NULL argument");
    return decode_stream(g->n, g->m, g->window, g->min_interval, g->bits.data(), g->nbits, row_ptr, col_idx);
}

extern "C" int bvg_bitstream_get(const bvg_host_graph* g, uint64_t* words, int64_t cap_words, int64_t* nbits) {
    if (!g || !nbits) return fail(BVG_ERR_INVALID_ARG, "bvg_bitstream_get: NULL argument");
    *nbits = g->nbits;
    if (!words) return BVG_OK;
    const int64_t need = (g->nbits + 63) / 64;
    if (cap_words < need) return fail(BVG_ERR_INVALID_ARG, "bvg_bitstream_get: %lld words needed", (long long)need);
    for (int64_t t = 0; t < need; t++) words[t] = g->bits[t];
    return BVG_OK;
}

extern "C" int bvg_decode_bits(int64_t n, int64_t m, const bvg_encode_params* params, const uint64_t* words,
                               int64_t nbits, int64_t* row_ptr, int32_t* col_idx) {
    if (n < 0 || m < 0 || nbits < 0 || !row_ptr || (m > 0 && !col_idx) || (nbits > 0 && !words))
        return fail(BVG_ERR_INVALID_ARG, "bvg_decode_bits: bad sizes or NULL arrays");
    const int W = params && params->window ? params->window : 7;
    const int L = params && params->min_interval ? params->min_interval : 4;
    if (W < 1 || W > kMaxWindow || L < 2) return fail(BVG_ERR_UNSUPPORTED, "bvg_decode_bits: window / min_interval");
    try {
        return decode_stream(n, m, W, L, words, nbits, row_ptr, col_idx);
    } catch (const std::bad_alloc&) {
        return fail(BVG_ERR_OOM, "bvg_decode_bits: host allocation failed");
    }
}

extern "C" int bvg_stats(const bvg_host_graph* g, bvg_graph_stats* out) {
    if (!g || !out) return fail(BVG_ERR_INVALID_ARG, "bvg_stats: NULL argument");
    *out = g->stats;
    return BVG_OK;
}

extern "C" int bvg_get_refs(const bvg_host_graph* g, int32_t* ref, int32_t* depth) {
    if (!g || !ref) return fail(BVG_ERR_INVALID_ARG, "bvg_get_refs: NULL argument");
    for (int64_t i = 0; i < g->n; i++) {
        ref[i] = g->ref[i];
        if (depth) depth[i] = g->depth[i];
    }
    return BVG_OK;
}

extern "C" int bvg_host_size(const bvg_host_graph* g, int64_t* n, int64_t* m) {
    if (!g) return fail(BVG_ERR_INVALID_ARG, "bvg_host_size: NULL graph");
    if (n) *n = g->n;
    if (m) *m = g->m;
    return BVG_OK;
}

extern "C" void bvg_free_host(bvg_host_graph* g) { delete g; }

extern "C" const char* bvg_status_string(int status) {
    switch (status) {
        case BVG_OK: return "ok";
        case BVG_ERR_INVALID_ARG: return "invalid argument";
        case BVG_ERR_BAD_GRAPH: return "bad graph (CSR not sorted, duplicate or out-of-range ids)";
        case BVG_ERR_OOM: return "out of memory";
        case BVG_ERR_CUDA: return "CUDA error";
        case BVG_ERR_NOT_CONVERGED: return "not converged within max_iter";
        case BVG_ERR_NUMERIC: return "non-finite value";
        case BVG_ERR_TIMEOUT: return "bounded device wait ran out";
        case BVG_ERR_CORRUPT: return "corrupt bitstream";
        case BVG_ERR_UNSUPPORTED: return "unsupported size or option";
        default: return "unknown status";
    }
}

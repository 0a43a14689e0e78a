// Biclique representation of a binary adjacency matrix (the second
// compressed format of the paper's final remarks, Sec. 6): the edges are
// split into bicliques (S_r, C_r), every node of S_r pointing to every node of
// C_r, stored as the two lists (|S_r| + |C_r| words for |S_r| * |C_r| edges),
// plus residual edges.
//
// The paper cites an extraction method without describing it; this file
// uses its own deterministic greedy miner:
//   - each pass hashes every remaining successor with a per-pass 64-bit mix
//     and keys each row by the smallest hash of its remaining successors (rows
//     with similar successor sets share the key with probability equal to
//     their Jaccard similarity);
//   - rows are ordered by (key, row) and each run of equal keys is scanned in
//     row order: a biclique starts from a row's remaining successors and takes
//     each of the next rows of the run (at most kScan of them) whose
//     intersection with it keeps the saving |S| * |C| - (|S| + |C|) from
//     shrinking;
//   - a biclique with at least two rows and a positive saving is emitted and
//     its edges leave the residual rows;
//   - finally, bicliques with the same column set are merged (their row sets
//     are disjoint, since the edges are), saving |C| words each: rows of one
//     block whose other successors gave them different keys end up together.
// Every step is in a fixed order, so the result depends only on the graph and
// the parameters.
#include <algorithm>
#include <new>
#include <vector>

#include "bvg_internal.h"


namespace {

constexpr int kScan = 64;  // rows of a key run a biclique looks ahead over

uint64_t mix64(uint64_t z) {  // splitmix64 finaliser
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

int64_t saving(int64_t s, int64_t c) { return s * c - (s + c); }

// Sorted intersection of two sorted lists.
void intersect(const std::vector<int32_t>& a, const std::vector<int32_t>& b, std::vector<int32_t>& out) {
    out.clear();
    std::set_intersection(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(out));
}

}  // namespace

using namespace bvg;

extern "C" int bvg_biclique_encode(int64_t n, const int64_t* row_ptr, const int32_t* col,
                                   const bvg_biclique_params* params, bvg_biclique** out) {
    if (!out) return fail(BVG_ERR_INVALID_ARG, "bvg_biclique_encode: out is NULL");
    *out = nullptr;
    if (n < 0 || n >= ((int64_t)1 << 31) || !row_ptr || (n > 0 && row_ptr[n] > 0 && !col))
        return fail(BVG_ERR_INVALID_ARG, "bvg_biclique_encode: bad n or NULL arrays");
    // defaults: 8 passes and 3 columns; on 200,000-row samples of the
    // generated graphs, 4 passes gave m/words 2.90 (web) and 1.21 (social),
    // 8 gave 3.01 and 1.23, 16 gave 3.03 and 1.24
    const int passes = params && params->passes > 0 ? params->passes : 8;
    const int64_t min_rows = params && params->min_rows > 1 ? params->min_rows : 2;
    const int64_t min_cols = params && params->min_cols > 1 ? params->min_cols : 3;
    const uint64_t seed = params ? params->seed : 0;
    if (row_ptr[0] != 0) return fail(BVG_ERR_INVALID_ARG, "bvg_biclique_encode: row_ptr[0] != 0");
    for (int64_t i = 0; i < n; i++) {
        if (row_ptr[i + 1] < row_ptr[i]) return fail(BVG_ERR_INVALID_ARG, "bvg_biclique_encode: row_ptr decreases");
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
            if (col[e] < 0 || col[e] >= n) return fail(BVG_ERR_INVALID_ARG, "bvg_biclique_encode: id out of range");
            if (e > row_ptr[i] && col[e] <= col[e - 1])
                return fail(BVG_ERR_INVALID_ARG, "bvg_biclique_encode: row %lld not sorted or repeats an id",
                            (long long)i);
        }
    }
    bvg_biclique* b = new (std::nothrow) bvg_biclique();
    if (!b) return fail(BVG_ERR_OOM, "bvg_biclique_encode: host allocation failed");
    try {
        b->n = n;
        b->m = n > 0 ? row_ptr[n] : 0;
        std::vector<std::vector<int32_t>> rest(n);
        for (int64_t i = 0; i < n; i++) rest[i].assign(col + row_ptr[i], col + row_ptr[i + 1]);
        std::vector<std::pair<uint64_t, int32_t>> keyed;
        std::vector<int32_t> cand, inter, group;
        std::vector<char> used;
        for (int p = 0; p < passes; p++) {
            const uint64_t salt = mix64(seed ^ (0x5bd1e995ull * (uint64_t)(p + 1)));
            keyed.clear();
            for (int64_t i = 0; i < n; i++) {
                if ((int64_t)rest[i].size() < min_cols) continue;
                uint64_t k = ~0ull;
                for (int32_t j : rest[i]) k = std::min(k, mix64((uint64_t)j ^ salt));
                keyed.push_back({k, (int32_t)i});
            }
            std::sort(keyed.begin(), keyed.end());
            for (size_t g0 = 0; g0 < keyed.size();) {
                size_t g1 = g0;
                while (g1 < keyed.size() && keyed[g1].first == keyed[g0].first) g1++;
                group.clear();
                for (size_t t = g0; t < g1; t++) group.push_back(keyed[t].second);
                used.assign(group.size(), 0);
                for (size_t a = 0; a < group.size(); a++) {
                    if (used[a] || (int64_t)rest[group[a]].size() < min_cols) continue;
                    std::vector<size_t> members{a};
                    cand = rest[group[a]];
                    for (size_t t = a + 1; t < group.size() && t <= a + kScan; t++) {
                        if (used[t]) continue;
                        intersect(cand, rest[group[t]], inter);
                        const int64_t s = (int64_t)members.size();
                        if ((int64_t)inter.size() >= min_cols &&
                            saving(s + 1, (int64_t)inter.size()) >= saving(s, (int64_t)cand.size())) {
                            members.push_back(t);
                            cand.swap(inter);
                        }
                    }
                    const int64_t s = (int64_t)members.size(), c = (int64_t)cand.size();
                    if (s < min_rows || saving(s, c) <= 0) continue;
                    std::vector<int32_t> rows;
                    for (size_t t : members) {
                        used[t] = 1;
                        rows.push_back(group[t]);
                    }
                    std::sort(rows.begin(), rows.end());
                    for (int32_t i : rows) {
                        std::vector<int32_t> left;
                        std::set_difference(rest[i].begin(), rest[i].end(), cand.begin(), cand.end(),
                                            std::back_inserter(left));
                        rest[i].swap(left);
                    }
                    b->s_idx.insert(b->s_idx.end(), rows.begin(), rows.end());
                    b->s_ptr.push_back((int64_t)b->s_idx.size());
                    b->c_idx.insert(b->c_idx.end(), cand.begin(), cand.end());
                    b->c_ptr.push_back((int64_t)b->c_idx.size());
                }
                g0 = g1;
            }
        }
        // merge bicliques with equal column sets (ordered by the sets, then by
        // first appearance, so the result stays deterministic)
        {
            const int64_t nb = (int64_t)b->s_ptr.size() - 1;
            std::vector<int64_t> order(nb);
            for (int64_t r = 0; r < nb; r++) order[r] = r;
            auto cbeg = [&](int64_t r) { return b->c_idx.begin() + b->c_ptr[r]; };
            auto cend = [&](int64_t r) { return b->c_idx.begin() + b->c_ptr[r + 1]; };
            std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) {
                return std::lexicographical_compare(cbeg(x), cend(x), cbeg(y), cend(y));
            });
            std::vector<int64_t> s_ptr{0}, c_ptr{0};
            std::vector<int32_t> s_idx, c_idx, rows;
            for (int64_t t = 0; t < nb;) {
                int64_t u = t;
                rows.clear();
                while (u < nb && std::equal(cbeg(order[t]), cend(order[t]), cbeg(order[u]), cend(order[u]))) {
                    rows.insert(rows.end(), b->s_idx.begin() + b->s_ptr[order[u]],
                                b->s_idx.begin() + b->s_ptr[order[u] + 1]);
                    u++;
                }
                std::sort(rows.begin(), rows.end());
                s_idx.insert(s_idx.end(), rows.begin(), rows.end());
                s_ptr.push_back((int64_t)s_idx.size());
                c_idx.insert(c_idx.end(), cbeg(order[t]), cend(order[t]));
                c_ptr.push_back((int64_t)c_idx.size());
                t = u;
            }
            b->s_ptr.swap(s_ptr);
            b->s_idx.swap(s_idx);
            b->c_ptr.swap(c_ptr);
            b->c_idx.swap(c_idx);
        }
        b->r_ptr.assign(n + 1, 0);
        for (int64_t i = 0; i < n; i++) b->r_ptr[i + 1] = b->r_ptr[i] + (int64_t)rest[i].size();
        b->r_col.reserve(b->r_ptr[n]);
        for (int64_t i = 0; i < n; i++) b->r_col.insert(b->r_col.end(), rest[i].begin(), rest[i].end());
    } catch (const std::bad_alloc&) {
        delete b;
        return fail(BVG_ERR_OOM, "bvg_biclique_encode: host allocation failed");
    }
    *out = b;
    return BVG_OK;
}

extern "C" int bvg_biclique_stats(const bvg_biclique* b, bvg_biclique_info* out) {
    if (!b || !out) return fail(BVG_ERR_INVALID_ARG, "bvg_biclique_stats: NULL argument");
    out->n = b->n;
    out->m = b->m;
    out->bicliques = (int64_t)b->s_ptr.size() - 1;
    out->s_total = (int64_t)b->s_idx.size();
    out->c_total = (int64_t)b->c_idx.size();
    out->residual = (int64_t)b->r_col.size();
    out->words = out->s_total + out->c_total + out->residual;
    int64_t covered = 0;
    for (int64_t r = 0; r < out->bicliques; r++)
        covered += (b->s_ptr[r + 1] - b->s_ptr[r]) * (b->c_ptr[r + 1] - b->c_ptr[r]);
    out->biclique_edges = covered;
    return BVG_OK;
}

extern "C" int bvg_biclique_get(const bvg_biclique* b, int64_t* s_ptr, int32_t* s_idx, int64_t* c_ptr,
                                int32_t* c_idx, int64_t* r_ptr, int32_t* r_col) {
    if (!b || !s_ptr || !c_ptr || !r_ptr || (!s_idx && !b->s_idx.empty()) || (!c_idx && !b->c_idx.empty()) ||
        (!r_col && !b->r_col.empty()))
        return fail(BVG_ERR_INVALID_ARG, "bvg_biclique_get: NULL array");
    std::copy(b->s_ptr.begin(), b->s_ptr.end(), s_ptr);
    std::copy(b->s_idx.begin(), b->s_idx.end(), s_idx);
    std::copy(b->c_ptr.begin(), b->c_ptr.end(), c_ptr);
    std::copy(b->c_idx.begin(), b->c_idx.end(), c_idx);
    std::copy(b->r_ptr.begin(), b->r_ptr.end(), r_ptr);
    std::copy(b->r_col.begin(), b->r_col.end(), r_col);
    return BVG_OK;
}

// Inverse memberships and the residual edges by column: the arrays a device
// product gathers from. row_bic[row_ptr2[i], row_ptr2[i + 1]) are the
// bicliques whose S holds row i (A x^T: y_i adds their c_r);
// col_bic[col_ptr2[j], col_ptr2[j + 1]) those whose C holds column j (x A: y_j
// adds their d_r); rt_row[rt_ptr[j], rt_ptr[j + 1]) the residual edges into
// column j, by source row. Every list is increasing.
extern "C" int bvg_biclique_gather_lists(const bvg_biclique* b, int64_t* row_ptr2, int32_t* row_bic, int64_t* col_ptr2,
                                         int32_t* col_bic, int64_t* rt_ptr, int32_t* rt_row) {
    if (!b || !row_ptr2 || !col_ptr2 || !rt_ptr || (!row_bic && !b->s_idx.empty()) ||
        (!col_bic && !b->c_idx.empty()) || (!rt_row && !b->r_col.empty()))
        return fail(BVG_ERR_INVALID_ARG, "bvg_biclique_gather_lists: NULL array");
    const int64_t n = b->n, nb = (int64_t)b->s_ptr.size() - 1;
    // counting sorts; bicliques and source rows are visited in increasing order
    std::fill(row_ptr2, row_ptr2 + n + 1, 0);
    std::fill(col_ptr2, col_ptr2 + n + 1, 0);
    std::fill(rt_ptr, rt_ptr + n + 1, 0);
    for (int32_t i : b->s_idx) row_ptr2[i + 1]++;
    for (int32_t j : b->c_idx) col_ptr2[j + 1]++;
    for (int32_t j : b->r_col) rt_ptr[j + 1]++;
    for (int64_t t = 0; t < n; t++) {
        row_ptr2[t + 1] += row_ptr2[t];
        col_ptr2[t + 1] += col_ptr2[t];
        rt_ptr[t + 1] += rt_ptr[t];
    }
    std::vector<int64_t> fr(row_ptr2, row_ptr2 + n), fc(col_ptr2, col_ptr2 + n), ft(rt_ptr, rt_ptr + n);
    for (int64_t r = 0; r < nb; r++) {
        for (int64_t e = b->s_ptr[r]; e < b->s_ptr[r + 1]; e++) row_bic[fr[b->s_idx[e]]++] = (int32_t)r;
        for (int64_t e = b->c_ptr[r]; e < b->c_ptr[r + 1]; e++) col_bic[fc[b->c_idx[e]]++] = (int32_t)r;
    }
    for (int64_t i = 0; i < n; i++)
        for (int64_t e = b->r_ptr[i]; e < b->r_ptr[i + 1]; e++) rt_row[ft[b->r_col[e]]++] = (int32_t)i;
    return BVG_OK;
}

extern "C" void bvg_free_biclique(bvg_biclique* b) { delete b; }

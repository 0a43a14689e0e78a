// Host construction of the device layout of a BV-delta encoding.
//
// desc[k]: bit t set iff row k + t + 1 is a descendant of row k in the
// reference forest (its chain passes through k); a chain spans at most kHalo
// rows, so kHalo bits suffice.
// Row-major difference rows (for A x^T): per row, 32-bit words tagged
// (two high bits) as dropped id, residual id, interval start + length word.
// Column-major entries (for x A): per column j, the source rows k whose
// difference row holds +1 or -1 at j, and interval events: an interval
// [s, e) of row k puts a start event at column s and an end event at column
// e (if e < n); the running sum of start - end events over columns is the
// interval part of y. Carry lists: for every tile of kCarryTile columns
// starting at a, the rows k of intervals with s < a <= e, whose start event
// lies before the tile and whose end event (if any) lies at or after a;
// summing their z gives the running sum at a without a grid-wide scan.
// Tail items: each column's entries past the first kGatherSlots, cut into
// runs of at most kTailItem entries (the gather hands them to its threads
// evenly instead of letting one thread walk a long column).
#include <algorithm>
#include <climits>
#include <new>

#include "bvg_internal.h"

namespace bvg {

int build_layout(const bvg_host_graph* hg, HostLayout& L) {
    const int64_t n = hg->n;
    const int64_t words = hg->stats.words;
    if (words >= ((int64_t)1 << 32)) return fail(BVG_ERR_UNSUPPORTED, "layout: more than 2^32 words");
    try {
        L.meta.assign(n, 0);
        L.desc.assign(n, 0);
        L.rowp.assign(n + 1, 0);
        L.ent.assign((size_t)words, 0);
        L.inv_outdeg.assign(n, 0.f);
        L.rowp[0] = 0;
        size_t w = 0;
        for (int64_t i = 0; i < n; i++) {
            const int off = hg->ref[i] >= 0 ? (int)(i - hg->ref[i]) : 0;
            L.meta[i] = (uint8_t)(off | (hg->depth[i] << kMetaDepthShift));
            // every ancestor r of i on its chain (at most kHalo rows back) gets
            // bit i - r - 1 of its descendant mask
            for (int64_t r = hg->ref[i], hop = 0; r >= 0 && hop < kMaxChain; r = hg->ref[r], hop++)
                L.desc[r] |= 1u << (i - r - 1);
            L.inv_outdeg[i] = hg->outdeg[i] ? 1.0f / (float)hg->outdeg[i] : 0.0f;
            for (int64_t t = hg->drop_ptr[i]; t < hg->drop_ptr[i + 1]; t++) L.ent[w++] = pack(kTagMinus, hg->drop[t]);
            for (int64_t t = hg->res_ptr[i]; t < hg->res_ptr[i + 1]; t++) L.ent[w++] = pack(kTagPlus, hg->res[t]);
            for (int64_t t = hg->iv_ptr[i]; t < hg->iv_ptr[i + 1]; t++) {
                L.ent[w++] = pack(kTagIvS, hg->iv_s[t]);
                L.ent[w++] = pack(kTagIvL, hg->iv_len[t]);
            }
            L.rowp[i + 1] = (uint32_t)w;
        }
        // ---- column-major entries (counting sort by column, rows in order)
        L.colp.assign(n + 1, 0);
        auto bump = [&](int64_t j) { L.colp[j + 1]++; };
        for (int64_t i = 0; i < n; i++) {
            for (int64_t t = hg->drop_ptr[i]; t < hg->drop_ptr[i + 1]; t++) bump(hg->drop[t]);
            for (int64_t t = hg->res_ptr[i]; t < hg->res_ptr[i + 1]; t++) bump(hg->res[t]);
            for (int64_t t = hg->iv_ptr[i]; t < hg->iv_ptr[i + 1]; t++) {
                bump(hg->iv_s[t]);
                int64_t e = (int64_t)hg->iv_s[t] + hg->iv_len[t];
                if (e < n) bump(e);
            }
        }
        for (int64_t j = 0; j < n; j++) {
            if ((int64_t)L.colp[j] + L.colp[j + 1] >= ((int64_t)1 << 32))
                return fail(BVG_ERR_UNSUPPORTED, "layout: more than 2^32 column entries");
            L.colp[j + 1] += L.colp[j];
        }
        if ((int64_t)L.colp[n] >= ((int64_t)1 << 30))
            return fail(BVG_ERR_UNSUPPORTED, "layout: more than 2^30 column entries");
        L.tent.assign(L.colp[n], 0);
        std::vector<uint32_t> fillp(L.colp.begin(), L.colp.end() - 1);
        const int64_t ntiles = (n + kCarryTile - 1) / kCarryTile;
        L.carry_ptr.assign(ntiles + 1, 0);
        for (int64_t i = 0; i < n; i++) {
            for (int64_t t = hg->drop_ptr[i]; t < hg->drop_ptr[i + 1]; t++)
                L.tent[fillp[hg->drop[t]]++] = pack(kTagMinus, (uint32_t)i);
            for (int64_t t = hg->res_ptr[i]; t < hg->res_ptr[i + 1]; t++)
                L.tent[fillp[hg->res[t]]++] = pack(kTagPlus, (uint32_t)i);
            for (int64_t t = hg->iv_ptr[i]; t < hg->iv_ptr[i + 1]; t++) {
                const int64_t s0 = hg->iv_s[t], e = s0 + hg->iv_len[t];
                L.tent[fillp[s0]++] = pack(kTagIvS, (uint32_t)i);
                if (e < n) L.tent[fillp[e]++] = pack(kTagIvL, (uint32_t)i);
                for (int64_t ct = s0 / kCarryTile + 1; ct <= e / kCarryTile && ct < ntiles; ct++) L.carry_ptr[ct + 1]++;
            }
        }
        for (int64_t t = 0; t < ntiles; t++) L.carry_ptr[t + 1] += L.carry_ptr[t];
        L.carry.assign(L.carry_ptr[ntiles], 0);
        std::vector<uint32_t> cfill(L.carry_ptr.begin(), L.carry_ptr.end() - 1);
        for (int64_t i = 0; i < n; i++)
            for (int64_t t = hg->iv_ptr[i]; t < hg->iv_ptr[i + 1]; t++) {
                const int64_t s0 = hg->iv_s[t], e = s0 + hg->iv_len[t];
                for (int64_t ct = s0 / kCarryTile + 1; ct <= e / kCarryTile && ct < ntiles; ct++)
                    L.carry[cfill[ct]++] = (uint32_t)i;
            }
        // tail items: each column's entries past the first kGatherSlots, in
        // runs of at most kTailItem
        L.titem_ptr.assign(n + 1, 0);
        for (int64_t j = 0; j < n; j++) {
            L.titem_ptr[j] = (uint32_t)L.titem.size();
            for (int64_t e = (int64_t)L.colp[j] + kGatherSlots; e < (int64_t)L.colp[j + 1]; e += kTailItem) {
                const int64_t cnt = std::min<int64_t>(kTailItem, (int64_t)L.colp[j + 1] - e);
                L.titem.push_back((uint32_t)e | (uint32_t)(cnt - 1) << 30);
            }
        }
        L.titem_ptr[n] = (uint32_t)L.titem.size();
    } catch (const std::bad_alloc&) {
        return fail(BVG_ERR_OOM, "layout: host allocation failed");
    }
    L.built = true;
    return BVG_OK;
}

// Pull work items: per row, the difference row with the intervals shorter
// than min_len expanded into single entries (a dropped id carries bit 31),
// cut into items of at most `item` consecutive entries; longer intervals are
// kept as (start, length). Rows of A' differ widely in length (exact copies
// have none, rows without a reference have all of theirs), so the pull
// parallelises over items of equal size, not over rows.
int build_pull_items(const uint32_t* rowp, const uint32_t* ent, int64_t n, int item, int min_len, PullItems& out,
                     bool only_if_worth) {
    if (item < 1) return fail(BVG_ERR_INVALID_ARG, "pull items: item < 1");
    if (only_if_worth) {
        // the prefix of x costs O(n) per product: keep intervals whole only
        // when their members outnumber 2n, else expand every one
        int64_t members = 0;
        for (int64_t q = 0; q < (int64_t)rowp[n]; q++)
            if ((ent[q] >> kIdBits) == kTagIvS) {
                const int64_t len = ent[q + 1] & kIdMask;
                if (len >= min_len) members += len;
                q++;
            }
        if (members <= 2 * n) min_len = INT32_MAX;
    }
    try {
        out = PullItems{};
        out.irow.assign(n + 1, 0);
        out.lrow.assign(n + 1, 0);
        out.pent.reserve((size_t)rowp[n] * 2);
        for (int64_t i = 0; i < n; i++) {
            const uint32_t b = (uint32_t)out.pent.size();
            out.irow[i] = (uint32_t)out.istart.size();
            out.lrow[i] = (uint32_t)(out.lint.size() / 2);
            for (uint32_t q = rowp[i]; q < rowp[i + 1]; q++) {
                const uint32_t w = ent[q], tag = w >> kIdBits, id = w & kIdMask;
                if (tag == kTagPlus) {
                    out.pent.push_back(id);
                } else if (tag == kTagMinus) {
                    out.pent.push_back(id | 0x80000000u);
                } else {
                    const uint32_t len = ent[++q] & kIdMask;
                    if ((int64_t)len >= min_len) {
                        out.lint.push_back(id);
                        out.lint.push_back(len);
                    } else {
                        for (uint32_t t = 0; t < len; t++) out.pent.push_back(id + t);
                    }
                }
                if (out.pent.size() >= ((size_t)1 << 32) - 1)
                    return fail(BVG_ERR_UNSUPPORTED, "pull items: more than 2^32 - 2 expanded entries");
            }
            for (uint32_t e = b; e < (uint32_t)out.pent.size(); e += (uint32_t)item) out.istart.push_back(e);
        }
        out.irow[n] = (uint32_t)out.istart.size();
        out.lrow[n] = (uint32_t)(out.lint.size() / 2);
        out.istart.push_back((uint32_t)out.pent.size());
    } catch (const std::bad_alloc&) {
        return fail(BVG_ERR_OOM, "pull items: host allocation failed");
    }
    return BVG_OK;
}

// Point columns: per column j, the source rows k whose difference row holds
// +1 (a residual id or a member of an interval) or -1 (a dropped id) at j,
// rows in increasing order, as kTagPlus / kTagMinus words. Unlike the event
// columns, an interval of length L costs L entries instead of two events,
// but the gather then needs no running interval sum across columns (no scan,
// no carry lists): y_j is the sum of column j's own entries. Tail items cut
// each column's entries past the first kPointSlots into runs of at most
// kTailItem.
int build_point_cols(const uint32_t* rowp, const uint32_t* ent, int64_t n, PointCols& out) {
    try {
        out = PointCols{};
        out.colp.assign(n + 1, 0);
        std::vector<int64_t> cnt(n + 1, 0);
        for (int64_t q = 0; q < (int64_t)rowp[n]; q++) {
            const uint32_t w = ent[q], tag = w >> kIdBits, id = w & kIdMask;
            if (tag == kTagPlus || tag == kTagMinus) {
                cnt[id + 1]++;
            } else {
                const uint32_t len = ent[++q] & kIdMask;
                for (uint32_t t = 0; t < len; t++) cnt[id + t + 1]++;
            }
        }
        for (int64_t j = 0; j < n; j++) cnt[j + 1] += cnt[j];
        if (cnt[n] >= ((int64_t)1 << 30)) return fail(BVG_ERR_UNSUPPORTED, "point columns: 2^30 entries or more");
        for (int64_t j = 0; j <= n; j++) out.colp[j] = (uint32_t)cnt[j];
        out.ent.assign((size_t)cnt[n], 0);
        for (int64_t i = 0; i < n; i++)
            for (uint32_t q = rowp[i]; q < rowp[i + 1]; q++) {
                const uint32_t w = ent[q], tag = w >> kIdBits, id = w & kIdMask;
                if (tag == kTagPlus || tag == kTagMinus) {
                    out.ent[cnt[id]++] = pack(tag, (uint32_t)i);
                } else {
                    const uint32_t len = ent[++q] & kIdMask;
                    for (uint32_t t = 0; t < len; t++) out.ent[cnt[id + t]++] = pack(kTagPlus, (uint32_t)i);
                }
            }
        out.titem_ptr.assign(n + 1, 0);
        for (int64_t j = 0; j < n; j++) {
            out.titem_ptr[j] = (uint32_t)out.titem.size();
            for (int64_t e = (int64_t)out.colp[j] + kPointSlots; e < (int64_t)out.colp[j + 1]; e += kTailItem) {
                const int64_t c = std::min<int64_t>(kTailItem, (int64_t)out.colp[j + 1] - e);
                out.titem.push_back((uint32_t)e | (uint32_t)(c - 1) << 30);
            }
        }
        out.titem_ptr[n] = (uint32_t)out.titem.size();
        out.long_chunk.assign((size_t)((n + kCarryTile - 1) / kCarryTile), 0);
        for (int64_t j = 0; j < n; j++)
            if ((int64_t)out.colp[j + 1] - out.colp[j] > (int64_t)kPointSlots + kLongColumn) out.long_chunk[j / kCarryTile] = 1;
    } catch (const std::bad_alloc&) {
        return fail(BVG_ERR_OOM, "point columns: host allocation failed");
    }
    return BVG_OK;
}

int get_layout(const bvg_host_graph* hg, const HostLayout** out) {
    std::lock_guard<std::mutex> lk(hg->layout_mu);
    if (!hg->layout) {
        HostLayout* L = new (std::nothrow) HostLayout();
        if (!L) return fail(BVG_ERR_OOM, "layout: host allocation failed");
        int rc = build_layout(hg, *L);
        if (rc) {
            delete L;
            return rc;
        }
        hg->layout.reset(L);
    }
    *out = hg->layout.get();
    return BVG_OK;
}

}  // namespace bvg

using namespace bvg;

extern "C" int bvg_layout_view_get(const bvg_host_graph* g, bvg_layout_view* out) {
    if (!g || !out) return fail(BVG_ERR_INVALID_ARG, "bvg_layout_view_get: NULL argument");
    const HostLayout* L = nullptr;
    int rc = get_layout(g, &L);
    if (rc) return rc;
    out->n = g->n;
    out->words = (int64_t)L->ent.size();
    out->col_entries = (int64_t)L->tent.size();
    out->carry_tiles = (int64_t)L->carry_ptr.size() - 1;
    out->carry_entries = (int64_t)L->carry.size();
    out->carry_tile_cols = kCarryTile;
    out->meta = L->meta.data();
    out->desc = L->desc.data();
    out->rowp = L->rowp.data();
    out->ent = L->ent.data();
    out->colp = L->colp.data();
    out->tent = L->tent.data();
    out->carry_ptr = L->carry_ptr.data();
    out->carry = L->carry.data();
    out->inv_outdeg = L->inv_outdeg.data();
    out->tail_items = (int64_t)L->titem.size();
    out->titem_ptr = L->titem_ptr.data();
    out->titem = L->titem.data();
    return BVG_OK;
}

extern "C" int bvg_pull_items_size(const bvg_host_graph* g, int32_t item, int32_t min_len, int64_t* entries,
                                   int64_t* items, int64_t* intervals) {
    if (!g || !entries || !items || !intervals || item < 1 || min_len < 1)
        return fail(BVG_ERR_INVALID_ARG, "bvg_pull_items_size: bad argument");
    const HostLayout* L = nullptr;
    int rc = get_layout(g, &L);
    if (rc) return rc;
    PullItems P;
    if ((rc = build_pull_items(L->rowp.data(), L->ent.data(), g->n, item, min_len, P, false))) return rc;
    *entries = (int64_t)P.pent.size();
    *items = (int64_t)P.istart.size() - 1;
    *intervals = (int64_t)P.lint.size() / 2;
    return BVG_OK;
}

extern "C" int bvg_pull_items_fill(const bvg_host_graph* g, int32_t item, int32_t min_len, uint32_t* pent,
                                   uint32_t* istart, uint32_t* irow, uint32_t* lrow, uint32_t* lint) {
    if (!g || !pent || !istart || !irow || !lrow || !lint || item < 1 || min_len < 1)
        return fail(BVG_ERR_INVALID_ARG, "bvg_pull_items_fill: bad argument");
    const HostLayout* L = nullptr;
    int rc = get_layout(g, &L);
    if (rc) return rc;
    PullItems P;
    if ((rc = build_pull_items(L->rowp.data(), L->ent.data(), g->n, item, min_len, P, false))) return rc;
    std::copy(P.pent.begin(), P.pent.end(), pent);
    std::copy(P.istart.begin(), P.istart.end(), istart);
    std::copy(P.irow.begin(), P.irow.end(), irow);
    std::copy(P.lrow.begin(), P.lrow.end(), lrow);
    std::copy(P.lint.begin(), P.lint.end(), lint);
    return BVG_OK;
}

extern "C" int bvg_point_cols_size(const bvg_host_graph* g, int64_t* entries, int64_t* tail_items) {
    if (!g || !entries || !tail_items) return fail(BVG_ERR_INVALID_ARG, "bvg_point_cols_size: NULL argument");
    const HostLayout* L = nullptr;
    int rc = get_layout(g, &L);
    if (rc) return rc;
    PointCols P;
    if ((rc = build_point_cols(L->rowp.data(), L->ent.data(), g->n, P))) return rc;
    *entries = (int64_t)P.ent.size();
    *tail_items = (int64_t)P.titem.size();
    return BVG_OK;
}

extern "C" int bvg_point_cols_fill(const bvg_host_graph* g, uint32_t* colp, uint32_t* ent, uint32_t* titem_ptr,
                                   uint32_t* titem) {
    if (!g || !colp || !ent || !titem_ptr || !titem) return fail(BVG_ERR_INVALID_ARG, "bvg_point_cols_fill: NULL argument");
    const HostLayout* L = nullptr;
    int rc = get_layout(g, &L);
    if (rc) return rc;
    PointCols P;
    if ((rc = build_point_cols(L->rowp.data(), L->ent.data(), g->n, P))) return rc;
    std::copy(P.colp.begin(), P.colp.end(), colp);
    std::copy(P.ent.begin(), P.ent.end(), ent);
    std::copy(P.titem_ptr.begin(), P.titem_ptr.end(), titem_ptr);
    std::copy(P.titem.begin(), P.titem.end(), titem);
    return BVG_OK;
}

// Autotuner: picks a device graph's launch configuration by timing the
// products with CUDA events, and keeps the choice in a JSON cache keyed by
// device, layout fingerprint and k.
//
// The searched space: the widest column block (k right-hand sides run as
// column blocks of at most this many), whether the push gather overlaps the
// chain kernel (programmatic dependent launch), the pull's entries per work
// item and rows per CTA of its row pass, and from which length on the pull
// keeps intervals unexpanded (summed from a prefix of x). Every setting gives the same products up to the product
// tolerance; only the time differs. Timing runs on warm caches (the
// configuration is chosen for repeated products, as in PageRank).
#include <cuda_runtime.h>

#include <algorithm>
#include <cctype>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "bvg_internal.h"

using namespace bvg;

namespace {

struct CacheEntry {
    bvg_launch_config cfg;
    double push_us = 0, pull_us = 0;
};

// ---- a small JSON reader for the cache's own format:
// {"version": 1, "entries": [{"key": "...", "pull_tile": 512, ...}, ...]}
struct Scanner {
    const std::string& s;
    size_t i = 0;
    explicit Scanner(const std::string& t) : s(t) {}
    void ws() {
        while (i < s.size() && std::isspace((unsigned char)s[i])) i++;
    }
    bool eat(char c) {
        ws();
        if (i < s.size() && s[i] == c) {
            i++;
            return true;
        }
        return false;
    }
    bool str(std::string& out) {
        ws();
        if (i >= s.size() || s[i] != '"') return false;
        out.clear();
        for (i++; i < s.size() && s[i] != '"'; i++) {
            if (s[i] == '\\') {
                if (++i >= s.size()) return false;
            }
            out.push_back(s[i]);
        }
        if (i >= s.size()) return false;
        i++;
        return true;
    }
    bool num(double& out) {
        ws();
        size_t j = i;
        while (j < s.size() && (std::isdigit((unsigned char)s[j]) || s[j] == '-' || s[j] == '+' || s[j] == '.' ||
                                s[j] == 'e' || s[j] == 'E'))
            j++;
        if (j == i) return false;
        try {
            out = std::stod(s.substr(i, j - i));
        } catch (...) {
            return false;
        }
        i = j;
        return true;
    }
};

bool parse_cache(const std::string& text, std::map<std::string, CacheEntry>& out) {
    Scanner sc(text);
    if (!sc.eat('{')) return false;
    bool seen_entries = false;
    while (true) {
        std::string name;
        if (!sc.str(name) || !sc.eat(':')) return false;
        if (name == "entries") {
            seen_entries = true;
            if (!sc.eat('[')) return false;
            if (!sc.eat(']')) {
                do {
                    if (!sc.eat('{')) return false;
                    std::string key;
                    CacheEntry e{};
                    e.cfg = {512, -1, 32, 1, 32, 8, -1, -1, -1};
                    int fields = 0;
                    do {
                        std::string f;
                        if (!sc.str(f) || !sc.eat(':')) return false;
                        if (f == "key") {
                            if (!sc.str(key)) return false;
                            continue;
                        }
                        double v = 0;
                        if (!sc.num(v)) return false;
                        if (f == "pull_tile") e.cfg.pull_tile = (int32_t)v, fields++;
                        else if (f == "pull_prefix") e.cfg.pull_prefix = (int32_t)v, fields++;
                        else if (f == "prefix_min_len") e.cfg.prefix_min_len = (int32_t)v, fields++;
                        else if (f == "gather_pdl") e.cfg.gather_pdl = (int32_t)v, fields++;
                        else if (f == "col_block") e.cfg.col_block = (int32_t)v, fields++;
                        else if (f == "pull_item") e.cfg.pull_item = (int32_t)v, fields++;
                        else if (f == "push_points") e.cfg.push_points = (int32_t)v;  // absent in older files: -1
                        else if (f == "push_fused") e.cfg.push_fused = (int32_t)v;    // absent in older files: -1
                        else if (f == "pull_fused") e.cfg.pull_fused = (int32_t)v;    // absent in older files: -1
                        else if (f == "push_us") e.push_us = v;
                        else if (f == "pull_us") e.pull_us = v;
                    } while (sc.eat(','));
                    if (!sc.eat('}') || key.empty() || fields != 6) return false;
                    out[key] = e;
                } while (sc.eat(','));
                if (!sc.eat(']')) return false;
            }
        } else {
            double v;
            std::string t;
            if (!sc.num(v) && !sc.str(t)) return false;
        }
        if (sc.eat(',')) continue;
        if (!sc.eat('}')) return false;
        break;
    }
    return seen_entries;
}

bool read_cache(const char* path, std::map<std::string, CacheEntry>& out) {
    std::ifstream f(path, std::ios::binary);
    if (!f) return false;
    std::stringstream ss;
    ss << f.rdbuf();
    std::map<std::string, CacheEntry> tmp;
    if (!parse_cache(ss.str(), tmp)) return false;
    out.swap(tmp);
    return true;
}

std::string json_escape(const std::string& s) {
    std::string o;
    for (char c : s) {
        if (c == '"' || c == '\\') o.push_back('\\');
        o.push_back(c);
    }
    return o;
}

int write_cache(const char* path, const std::map<std::string, CacheEntry>& m) {
    std::ostringstream o;
    o << "{\"version\": 1, \"entries\": [";
    bool first = true;
    for (const auto& kv : m) {  // keys in sorted order
        const bvg_launch_config& c = kv.second.cfg;
        char buf[512];
        std::snprintf(buf, sizeof buf,
                      "%s\n  {\"key\": \"%s\", \"pull_tile\": %d, \"pull_prefix\": %d, \"prefix_min_len\": %d, "
                      "\"gather_pdl\": %d, \"col_block\": %d, \"pull_item\": %d, \"push_points\": %d, "
                      "\"push_fused\": %d, \"pull_fused\": %d, \"push_us\": %.3f, \"pull_us\": %.3f}",
                      first ? "" : ",", json_escape(kv.first).c_str(), c.pull_tile, c.pull_prefix, c.prefix_min_len,
                      c.gather_pdl, c.col_block, c.pull_item, c.push_points, c.push_fused, c.pull_fused,
                      kv.second.push_us,
                      kv.second.pull_us);
        o << buf;
        first = false;
    }
    o << "\n]}\n";
    const std::string tmp = std::string(path) + ".tmp";
    {
        std::ofstream f(tmp, std::ios::binary | std::ios::trunc);
        if (!f) return fail(BVG_ERR_INVALID_ARG, "autotune cache: cannot write %s", tmp.c_str());
        f << o.str();
        if (!f) return fail(BVG_ERR_INVALID_ARG, "autotune cache: write to %s failed", tmp.c_str());
    }
    if (std::rename(tmp.c_str(), path) != 0) return fail(BVG_ERR_INVALID_ARG, "autotune cache: rename to %s failed", path);
    return BVG_OK;
}

int make_key(const bvg_dev_graph* g, int k, std::string& key) {
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, g->device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(BVG_ERR_CUDA, "bvg_autotune: %s", cudaGetErrorString(e));
    }
    std::string name = prop.name;
    for (char& c : name)
        if (!std::isalnum((unsigned char)c)) c = '_';
    char buf[256];
    std::snprintf(buf, sizeof buf, "%s/sm%d/%016llx/k%d", name.c_str(), prop.multiProcessorCount,
                  (unsigned long long)g->fingerprint, k);
    key = buf;
    return BVG_OK;
}

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    Timer() {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~Timer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

// Median of `reps` timed calls after `warm` untimed ones (microseconds), or
// a negative status.
template <class F>
int time_op(F op, cudaStream_t st, Timer& t, double* us) {
    const int warm = 2, reps = 7;
    for (int i = 0; i < warm; i++) {
        int rc = op();
        if (rc) return rc;
    }
    std::vector<double> v;
    for (int i = 0; i < reps; i++) {
        cudaEventRecord(t.a, st);
        int rc = op();
        if (rc) return rc;
        cudaEventRecord(t.b, st);
        cudaError_t e = cudaEventSynchronize(t.b);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(BVG_ERR_CUDA, "bvg_autotune: %s", cudaGetErrorString(e));
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, t.a, t.b);
        v.push_back(1e3 * ms);
    }
    std::sort(v.begin(), v.end());
    *us = v[v.size() / 2];
    return BVG_OK;
}

}  // namespace

extern "C" int bvg_autotune_key(const bvg_dev_graph* g, int32_t k, char* buf, int32_t cap) {
    if (!g || !buf || cap < 1 || k < 1) return fail(BVG_ERR_INVALID_ARG, "bvg_autotune_key: bad argument");
    std::string key;
    int rc = make_key(g, k, key);
    if (rc) return rc;
    if ((int32_t)key.size() + 1 > cap) return fail(BVG_ERR_INVALID_ARG, "bvg_autotune_key: buffer too small");
    std::memcpy(buf, key.c_str(), key.size() + 1);
    return BVG_OK;
}

extern "C" int bvg_autotune_cache_lookup(const char* path, const char* key, bvg_launch_config* out, int32_t* found) {
    if (!path || !key || !out || !found) return fail(BVG_ERR_INVALID_ARG, "bvg_autotune_cache_lookup: NULL argument");
    *found = 0;
    std::map<std::string, CacheEntry> m;
    if (!read_cache(path, m)) return BVG_OK;  // missing or unreadable: nothing cached
    auto it = m.find(key);
    if (it == m.end()) return BVG_OK;
    *out = it->second.cfg;
    *found = 1;
    return BVG_OK;
}

extern "C" int bvg_autotune_cache_store(const char* path, const char* key, const bvg_launch_config* cfg,
                                        double push_us, double pull_us) {
    if (!path || !key || !cfg || !*key) return fail(BVG_ERR_INVALID_ARG, "bvg_autotune_cache_store: bad argument");
    std::map<std::string, CacheEntry> m;
    read_cache(path, m);  // a missing or corrupt file starts a new cache
    CacheEntry e;
    e.cfg = *cfg;
    e.push_us = push_us;
    e.pull_us = pull_us;
    m[key] = e;
    return write_cache(path, m);
}

extern "C" int bvg_autotune(bvg_dev_graph* g, int32_t k, const char* cache_path, void* stream) {
    if (!g || k < 1) return fail(BVG_ERR_INVALID_ARG, "bvg_autotune: need a graph and k >= 1");
    g->tune = TuneInfo{};
    if (g->n == 0) return BVG_OK;
    cudaStream_t st = (cudaStream_t)stream;
    std::string key;
    int rc = make_key(g, k, key);
    if (rc) return rc;
    bvg_launch_config base;
    if ((rc = bvg_get_config(g, &base))) return rc;
    if (cache_path) {
        bvg_launch_config c;
        int32_t found = 0;
        if ((rc = bvg_autotune_cache_lookup(cache_path, key.c_str(), &c, &found))) return rc;
        if (found && bvg_set_config(g, &c) == BVG_OK) {
            g->tune.from_cache = 1;
            return BVG_OK;
        }
    }
    // scratch right-hand sides: 0x3f3f3f3f = 0.747 in every entry
    float *x = nullptr, *y = nullptr;
    const size_t bytes = (size_t)g->n * k * sizeof(float);
    if (cudaMalloc(&x, bytes) != cudaSuccess || cudaMalloc(&y, bytes) != cudaSuccess) {
        cudaGetLastError();
        if (x) cudaFree(x);
        return fail(BVG_ERR_OOM, "bvg_autotune: scratch allocation failed");
    }
    auto release = [&]() {
        cudaStreamSynchronize(st);
        cudaFree(x);
        cudaFree(y);
    };
    if (cudaMemsetAsync(x, 0x3f, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        release();
        return fail(BVG_ERR_CUDA, "bvg_autotune: memset failed");
    }
    Timer t;
    auto push = [&]() { return bvg_spmv_xA(g, x, y, k, k, st); };
    auto pull = [&]() { return bvg_spmv_Ax(g, x, y, k, k, st); };
    int kpow = 1;
    while (kpow * 2 <= std::min(k, 32)) kpow *= 2;
    // push: column block x overlap x gather over event or point columns
    bvg_launch_config best = base;
    double best_push = 1e300;
    if ((rc = time_op(push, st, t, &g->tune.push_us_default))) {
        release();
        return rc;
    }
    // one right-hand side: the fused kernel too (which has no overlap or column layout to choose)
    const int fz_lo = kpow == 1 ? 0 : -1, fz_hi = kpow == 1 ? 1 : -1;
    for (int fz = fz_lo; fz <= fz_hi; fz++)
    for (int cb = kpow; cb >= std::max(1, kpow / 8); cb >>= 1) {
        for (int pdl = 0; pdl <= 1; pdl++)
            for (int pts = 0; pts <= 1; pts++) {
                if (fz == 1 && (pdl == 0 || pts == 0)) continue;
                bvg_launch_config c = base;
                c.col_block = cb;
                c.gather_pdl = pdl;
                c.push_points = pts;
                c.push_fused = fz;
                double us = 0;
                if ((rc = bvg_set_config(g, &c)) || (rc = time_op(push, st, t, &us))) {
                    bvg_set_config(g, &base);
                    release();
                    return rc;
                }
                g->tune.candidates++;
                if (us < best_push) {
                    best_push = us;
                    best = c;
                }
            }
    }
    // pull: entries per work item x rows per CTA of the row pass x which
    // intervals stay unexpanded (summed from the prefix), with the chosen column block
    bvg_launch_config b2 = best;
    if ((rc = bvg_set_config(g, &b2)) || (rc = time_op(pull, st, t, &g->tune.pull_us_default))) {
        bvg_set_config(g, &base);
        release();
        return rc;
    }
    double best_pull = 1e300;
    // one right-hand side: the one-launch pull where every row tile fits it
    // (it has no item size, tile or interval rule to choose), against the
    // two-kernel pull's settings below
    const bool px = kpow == 1 && g->px_ok;
    if (px) {
        bvg_launch_config c = best;
        c.pull_fused = 1;
        double us = 0;
        if ((rc = bvg_set_config(g, &c)) || (rc = time_op(pull, st, t, &us))) {
            bvg_set_config(g, &base);
            release();
            return rc;
        }
        g->tune.candidates++;
        best_pull = us;
        b2 = c;
    }
    std::vector<int> minlens = {32};
    if (g->mean_interval > 0) minlens.insert(minlens.end(), {16, 1 << 20});  // 1 << 20: expand every interval
    for (int ml : minlens) {
        for (int item : {4, 8, 16}) {
            for (int tile : {256, 512}) {
                bvg_launch_config c = best;
                c.pull_tile = tile;
                c.pull_item = item;
                c.prefix_min_len = ml;
                c.pull_prefix = -1;
                if (px) c.pull_fused = 0;
                double us = 0;
                if ((rc = bvg_set_config(g, &c)) || (rc = time_op(pull, st, t, &us))) {
                    bvg_set_config(g, &base);
                    release();
                    return rc;
                }
                g->tune.candidates++;
                if (us < best_pull) {
                    best_pull = us;
                    b2 = c;
                }
            }
        }
    }
    release();
    if ((rc = bvg_set_config(g, &b2))) return rc;
    g->tune.push_us_best = best_push;
    g->tune.pull_us_best = best_pull;
    if (cache_path) return bvg_autotune_cache_store(cache_path, key.c_str(), &b2, best_push, best_pull);
    return BVG_OK;
}

extern "C" int bvg_autotune_info_get(const bvg_dev_graph* g, bvg_autotune_info* out) {
    if (!g || !out) return fail(BVG_ERR_INVALID_ARG, "bvg_autotune_info_get: NULL argument");
    out->from_cache = g->tune.from_cache;
    out->candidates = g->tune.candidates;
    out->push_us_default = g->tune.push_us_default;
    out->push_us_best = g->tune.push_us_best;
    out->pull_us_default = g->tune.pull_us_default;
    out->pull_us_best = g->tune.pull_us_best;
    return BVG_OK;
}

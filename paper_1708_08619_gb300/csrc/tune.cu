// Autotuner for the tensor-core band kernel's free parameters:
//   kseg       -- K elements per work item (more items balance the grid
//                 better, fewer items pay fewer end-of-item reductions, and
//                 shorter items keep the operand rows of the items in flight
//                 in L2);
//   supertile  -- the claim order of the band tiles: super_rows row tiles x
//                 super_cols column tiles at a time, which sets how the ~152
//                 items in flight share A and B rows in L2;
//   tile shape -- 128 x 192 tiles on one CTA each, or 256 x 192 on a CTA pair
//                 (cta_group::2, each CTA loading its A tile and half of B);
//   sub_kb     -- K-blocks per TMEM accumulation sub-chain (longer chains
//                 hand the accumulator over less often but lose more low bits).
// kseg, the supertile and the tile shape are timed; sub_kb decides the accuracy, so the
// candidates leave it at 0, which stands for the kind's default (a cached
// nonzero sub_kb, written by hand or by an older library, is honoured).
// Without TCORR_TUNE the library uses defaults measured on GB300
// (tune_default_kseg, a 16 x 10 supertile, one-CTA tiles).  With TCORR_TUNE=1 the first
// call for a shape bucket times every candidate on the caller's stream (this
// synchronises, so it is skipped while the stream is being captured) and
// remembers the fastest; TCORR_TUNE=force re-times on every call.
// TCORR_TUNE_CACHE names a file of JSON lines {"key": ..., "kseg": ...,
// "sub_kb": ..., "super_rows": ..., "super_cols": ..., "pair": ...} that is
// read at the first lookup and appended to after each tuning run (lines
// without the supertile or tile-shape fields are read with the defaults).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "tcorr_internal.cuh"

namespace tcorr {
namespace {

std::mutex g_tune_mu;
std::map<std::string, TuneChoice> g_tune;
bool g_tune_loaded = false;
thread_local const TuneChoice *g_override = nullptr;

int ilog2_ceil(int64_t v) {
    int b = 0;
    while ((int64_t(1) << b) < v && b < 62) ++b;
    return b;
}

void load_cache_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = std::getenv("TCORR_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char line[512];
    while (std::fgets(line, sizeof line, f)) {
        char key[256];
        long long kseg = 0;
        int sub = 0, sr = 0, sc = 0, pr = -1;
        const int got = std::sscanf(line, " {\"key\": \"%255[^\"]\", \"kseg\": %lld, \"sub_kb\": %d, "
                                          "\"super_rows\": %d, \"super_cols\": %d, \"pair\": %d",
                                    key, &kseg, &sub, &sr, &sc, &pr);
        if (got >= 3 && kseg >= 64 && sub >= 0) {
            TuneChoice c{kseg, sub};
            if (got >= 5 && sr >= 1 && sc >= 1 && sr <= 4096 && sc <= 4096) {
                c.super_rows = sr;
                c.super_cols = sc;
            }
            if (got == 6 && (pr == 0 || pr == 1)) c.pair = pr;
            g_tune[key] = c;
        }
    }
    std::fclose(f);
}

}  // namespace

int tune_mode() {
    const char *e = std::getenv("TCORR_TUNE");
    if (!e || !*e || std::strcmp(e, "0") == 0) return 0;
    return std::strcmp(e, "force") == 0 ? 2 : 1;
}

std::string tune_key(int method, int kind, int64_t K, int64_t tau_max, int64_t T, int64_t s) {
    char buf[128];
    std::snprintf(buf, sizeof buf, "m%d.k%d.K%d.tm%d.T%d.s%d", method, kind, ilog2_ceil(K),
                  ilog2_ceil(tau_max + 1), ilog2_ceil(T), static_cast<int>(s < 4 ? s : 4));
    return buf;
}

bool tune_lookup(const std::string &key, TuneChoice *c) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    load_cache_locked();
    const auto it = g_tune.find(key);
    if (it == g_tune.end()) return false;
    *c = it->second;
    return true;
}

void tune_store(const std::string &key, const TuneChoice &c) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    load_cache_locked();
    g_tune[key] = c;
    if (const char *path = std::getenv("TCORR_TUNE_CACHE")) {
        if (FILE *f = std::fopen(path, "a")) {
            std::fprintf(f, "{\"key\": \"%s\", \"kseg\": %lld, \"sub_kb\": %d, \"super_rows\": %d, "
                            "\"super_cols\": %d, \"pair\": %d}\n",
                         key.c_str(), static_cast<long long>(c.kseg), c.sub_kb, c.super_rows, c.super_cols,
                         c.pair < 0 ? 0 : c.pair);
            std::fclose(f);
        }
    }
}

const std::vector<TuneChoice> &tune_candidates() {
    static const std::vector<TuneChoice> c = [] {
        std::vector<TuneChoice> v;
        const int shapes[3][2] = {{16, 10}, {32, 5}, {8, 19}};
        for (int pair : {0, 1})
            for (int64_t kseg : {4096, 8192, 16384})
                for (const auto &sh : shapes) {
                    TuneChoice t{kseg, 0};
                    t.super_rows = sh[0];
                    t.super_cols = sh[1];
                    t.pair = pair;
                    v.push_back(t);
                }
        return v;
    }();
    return c;
}

int64_t tune_min_kseg() { return 4096; }

void set_tune_override(const TuneChoice *c) { g_override = c; }
const TuneChoice *get_tune_override() { return g_override; }

// Work-item length: long items (fewer end-of-item reductions) unless the
// band has too few tiles to give every SM several items, and at most 8192
// K elements when a band row has 24 column tiles or more.  Measured on GB300
// (16 x 10 supertiles, FP16x3): water scale (12 column tiles per row) took
// 6.93 / 7.27 / 8.02 ms per MSD launch at 16384 / 8192 / 4096 elements; the
// precision workload (53 per row) 213 / 208 / 216 ms, its autocorrelation
// 234 / 221 / 222 ms.
int64_t tune_default_kseg(int64_t K, int64_t tiles, int64_t n_cols) {
    const int64_t want_items = 4 * 152;
    int64_t kseg = ceil_div(K * tiles, want_items);
    kseg = ceil_div(kseg, 512) * 512;
    if (kseg < 512) kseg = 512;
    const int64_t cap = n_cols >= 24 ? 8192 : 16384;
    if (kseg > cap) kseg = cap;
    return kseg;
}

}  // namespace tcorr

// Autotuner for the tensor-core band kernel's two free parameters:
//   kseg   -- K elements per work item (more items balance the grid better,
//             fewer items pay fewer end-of-item reductions);
//   sub_kb -- K-blocks per TMEM accumulation sub-chain (longer chains hand
//             the accumulator over less often but lose more low bits).
// Only kseg is timed: sub_kb decides the accuracy, so the candidates leave it
// at 0, which stands for the kind's default (a cached nonzero sub_kb, written
// by hand or by an older library, is honoured).  Without TCORR_TUNE the
// library uses a heuristic (tune_default_kseg).  With TCORR_TUNE=1 the first call for a shape
// bucket times every candidate on the caller's stream (this synchronises,
// so it is skipped while the stream is being captured) and remembers the
// fastest; TCORR_TUNE=force re-times on every call.  TCORR_TUNE_CACHE names
// a file of JSON lines {"key": ..., "kseg": ..., "sub_kb": ...} that is read
// at the first lookup and appended to after each tuning run.
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
        int sub = 0;
        if (std::sscanf(line, " {\"key\": \"%255[^\"]\", \"kseg\": %lld, \"sub_kb\": %d", key, &kseg, &sub) == 3 &&
            kseg >= 64 && sub >= 1)
            g_tune[key] = TuneChoice{kseg, sub};
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
            std::fprintf(f, "{\"key\": \"%s\", \"kseg\": %lld, \"sub_kb\": %d}\n", key.c_str(),
                         static_cast<long long>(c.kseg), c.sub_kb);
            std::fclose(f);
        }
    }
}

const std::vector<TuneChoice> &tune_candidates() {
    static const std::vector<TuneChoice> c = {{4096, 0}, {8192, 0}, {16384, 0}};
    return c;
}

int64_t tune_min_kseg() { return 4096; }

void set_tune_override(const TuneChoice *c) { g_override = c; }
const TuneChoice *get_tune_override() { return g_override; }

// Work-item length: long items (fewer end-of-item reductions) unless the
// band has too few tiles to give every SM several items.
int64_t tune_default_kseg(int64_t K, int64_t tiles) {
    const int64_t want_items = 4 * 152;
    int64_t kseg = ceil_div(K * tiles, want_items);
    kseg = ceil_div(kseg, 512) * 512;
    if (kseg < 512) kseg = 512;
    if (kseg > 16384) kseg = 16384;
    return kseg;
}

}  // namespace tcorr

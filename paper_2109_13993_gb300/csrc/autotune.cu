// autotune.cu -- the pair-tile autotuner: the tile rows (64 or 32) of the mixed path
// per problem-size bucket (ceil(log2 p), ceil(log2 n)), measured by lingam_autotune on
// the caller's data and kept in a process-wide table; buckets never measured use a
// default rule.
#include <chrono>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "launch.h"
#include "lingam.h"

namespace lingam {

static std::mutex g_tune_mu;
static std::map<std::pair<int, int>, int> g_tune;   // (p bucket, n bucket) -> tile rows

static int ceil_log2(long long v) {
    int b = 0;
    while ((1ll << b) < v) ++b;
    return b;
}

static std::pair<int, int> bucket(long long p, long long n) { return {ceil_log2(p), ceil_log2(n)}; }

// Default when a bucket was never measured: 64-row tiles, measured faster than
// 32-row tiles for single fits of p = 20 ... 1000 at n = 2000 and 10^4 on GB300
// (by 6 % at p = 1000 to 31 % at p = 50).
static int default_tile_rows(long long p, long long n) {
    (void)p;
    (void)n;
    return 64;
}

int autotune_tile_rows(long long p, long long n) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(bucket(p, n));
    return it != g_tune.end() ? it->second : default_tile_rows(p, n);
}

void autotune_record(long long p, long long n, int tile_rows) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[bucket(p, n)] = tile_rows;
}

void autotune_clear() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
}

}  // namespace lingam

// autotune.cu -- the pair-tile autotuner: the tile shape (rows x columns: 64 x 32,
// 32 x 32 or 64 x 16) of the mixed path per problem-size bucket (ceil(log2 p),
// ceil(log2 n)), measured by lingam_autotune (single fits) or lingam_autotune_batch
// (batch calls, bucket of the largest p and n) on the caller's data and kept in two
// process-wide tables; buckets never measured use a default rule.
#include <chrono>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "launch.h"
#include "lingam.h"

namespace lingam {

static std::mutex g_tune_mu;
static std::map<std::pair<int, int>, TileShape> g_tune;   // (p bucket, n bucket) -> shape

static int ceil_log2(long long v) {
    int b = 0;
    while ((1ll << b) < v) ++b;
    return b;
}

static std::pair<int, int> bucket(long long p, long long n) { return {ceil_log2(p), ceil_log2(n)}; }

// Default when a bucket was never measured: 64 x 32 tiles, measured faster than
// 32 x 32 tiles for single fits of p = 20 ... 1000 at n = 2000 and 10^4 on GB300
// (by 6 % at p = 1000 to 31 % at p = 50).
static TileShape default_tile_shape(long long p, long long n) {
    (void)p;
    (void)n;
    return TileShape{64, 32};
}

TileShape autotune_tile_shape(long long p, long long n) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(bucket(p, n));
    return it != g_tune.end() ? it->second : default_tile_shape(p, n);
}

void autotune_record(long long p, long long n, TileShape shape) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[bucket(p, n)] = shape;
}

// Batch calls: a table of its own, keyed by the batch's largest p and n.  Default: 32 x 32
// tiles, which a batch of many small problems pads least once r < 32.
static std::map<std::pair<int, int>, TileShape> g_tune_batch;

TileShape autotune_batch_shape(long long maxp, long long maxn) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_batch.find(bucket(maxp, maxn));
    if (it != g_tune_batch.end()) return it->second;
    // never measured: the pair-per-warp mode up to 128 variables (it wins over every tile
    // shape on the measured batches of small problems), else 32 x 32
    return maxp <= 128 ? TileShape{1, 1} : TileShape{32, 32};
}

void autotune_batch_record(long long maxp, long long maxn, TileShape shape) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_batch[bucket(maxp, maxn)] = shape;
}

void autotune_clear() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
    g_tune_batch.clear();
}

}  // namespace lingam

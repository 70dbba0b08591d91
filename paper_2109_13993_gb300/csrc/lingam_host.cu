// lingam_host.cu -- the C ABI of include/lingam.h: argument checks, workspace
// layout, the launch sequence of Algorithm 3 on one stream, and the copies of
// the results.  The library allocates no memory: every buffer is carved out
// of the caller's workspace.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>

#include "common.cuh"
#include "launch.h"
#include "lingam.h"

namespace lingam {

cudaError_t ensure_smem_attr(const void* func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(func, dev);
    auto it = done.find(key);
    if (it != done.end() && it->second >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (e == cudaSuccess) done[key] = bytes;
    return e;
}

constexpr long long kMaxP = 16384;
constexpr size_t kAlign = 256;

static size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Host-side fault injection for tests of the error paths (no GPU fault is involved):
// the environment variable LINGAM_FAULT names a step of a call -- "standardize",
// "covariance", "iteration" (optionally "iteration:<k>" for iteration k), "bfit" or "batch"
// -- and that step reports a failed launch (LINGAM_ECUDA) instead of launching.
static bool inject_fault(const char* step, int k = -1) {
    const char* e = std::getenv("LINGAM_FAULT");
    if (!e || !*e) return false;
    const size_t n = std::strlen(step);
    if (std::strncmp(e, step, n) != 0) return false;
    if (e[n] == '\0') return true;
    return e[n] == ':' && k >= 0 && std::atoi(e + n + 1) == k;
}

// LINGAM_LOG >= 1: one line per call on stderr (sizes, status, launches, device times).
static int log_level() {
    const char* e = std::getenv("LINGAM_LOG");
    return e ? std::atoi(e) : 0;
}

struct Layout {
    size_t total = 0;
    size_t off_xin, off_xt, off_mu, off_sd, off_sig, off_sig0, off_sigf, off_hx, off_vstat, off_part, off_cflag, off_crow, off_prev, off_flags,
        off_sigma, off_sigma_alt,
        off_rows, off_cols, off_order, off_forced, off_prior, off_anc, off_scratch, off_rowsum, off_colsum, off_partials, off_invroot,
        off_tilecnt, off_rs, off_rm, off_rp, off_rsc, off_cmat, off_rmat, off_rinv, off_bout, off_ctl, off_ibuf;
    int ld, maxtiles, maxsplit, esz, nslots;
};

static int chunk_of(int precision) { return precision == LINGAM_MIXED ? kChunk : kChunk64; }

static Layout make_layout(long long p, long long n, int precision, int input_dtype, bool with_prior = false) {
    Layout L;
    L.ld = int((n + kSampleAlign - 1) / kSampleAlign * kSampleAlign);
    L.esz = precision == LINGAM_MIXED ? 4 : 8;
    L.maxtiles = int((p + kTI - 1) / kTI);
    L.maxsplit = std::max(1, std::min(kMaxSplit, L.ld / chunk_of(precision)));
    const size_t in_esz = input_dtype == LINGAM_F32 ? 4 : 8;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    const size_t P = size_t(p), PP = size_t(p) * size_t(p);
    L.off_ctl = take(sizeof(Ctl));
    // the host-input copy is dead once the rows are normalised; the mixed path's
    // tensor-core Gram reuses it for the digit planes of its operands
    const size_t split_bytes = precision == LINGAM_MIXED ? gram_tc_digit_bytes(p, L.ld) : 0;
    L.off_xin = take(std::max(P * size_t(n) * in_esz, split_bytes));
    L.off_xt = take(P * size_t(L.ld) * L.esz);
    L.off_mu = take(P * 8);
    L.off_sd = take(P * 8);
    L.off_sig = take(PP * 8);
    L.off_sig0 = take(PP * 8);
    L.off_sigf = take(precision == LINGAM_MIXED ? PP * 8 : 0);
    L.off_hx = take(P * 8);
    L.off_vstat = take(P * 16);
    L.off_part = take(P * 8);
    L.off_cflag = take(P * 4);
    L.off_crow = take(P * 4);
    L.off_prev = take(P * 8);
    L.off_flags = take(P * 4);
    L.off_sigma = take(P * 4);
    L.off_sigma_alt = take(P * 4);
    L.off_rows = take(P * 4);
    L.off_cols = take(kTJ * 4);
    L.off_order = take(P * 4);
    L.off_forced = take(P * 4);
    L.off_prior = take(with_prior ? PP : 0);
    L.off_anc = take(with_prior ? P * 4 : 0);
    L.off_scratch = take(P * 4);
    L.off_rowsum = take(P * 8);
    L.off_colsum = take(size_t(L.maxtiles) * (kPairThreads / 64) * kTJ * 8);   // per (tile, merge item)
    // one partial-moment slot per (tile, CTA) segment; slot index tile + CTA, and a wave never
    // uses more CTAs than it has (tile, 32-sample group) units
    const size_t units = size_t(L.maxtiles) * size_t(L.ld / kSub);
    // (the Gram's split partial tiles use the same region before the first iteration)
    L.nslots = int(size_t(L.maxtiles) + std::min(size_t(kMaxGrid), units));
    const size_t pair_partials = size_t(L.nslots) * kPairThreads * 16 * L.esz;
    L.off_partials =
        take(std::max(pair_partials, precision == LINGAM_MIXED ? gram_tc_partial_bytes(p, L.ld) : size_t(0)));
    L.off_invroot = take(P * 8);
    L.off_tilecnt = take(size_t(L.maxtiles) * 4);
    L.off_ibuf = take(size_t(L.maxtiles) * 64 * kTJ * L.esz);
    L.off_rs = take(P * 8);
    L.off_rm = take(P * 8);
    L.off_rp = take(P * 8);
    L.off_rsc = take(PP * 8);
    L.off_cmat = take(PP * 8);
    L.off_rmat = take(PP * 8);
    L.off_rinv = take(PP * 8);
    L.off_bout = take(PP * 8);
    L.total = o;
    return L;
}

// Pair-tile shape of the mixed path: the caller's choice (tile_i rows, tile_j columns;
// a zero takes 64 rows or 32 columns), else the tile autotuner's choice for this size.
static TileShape choose_tile(long long p, long long n, int tile_i, int tile_j) {
    if (tile_i == 0 && tile_j == 0) return autotune_tile_shape(p, n);
    return TileShape{tile_i ? tile_i : 64, tile_j ? tile_j : 32};
}

static bool valid_opts(const lingam_opts& o) {
    return (o.precision == LINGAM_MIXED || o.precision == LINGAM_FP64) &&
           (o.input_dtype == LINGAM_F32 || o.input_dtype == LINGAM_F64) && (o.prune == 0 || o.prune == 1) &&
           (o.reuse == 0 || o.reuse == 1) && o.split_n >= 0 &&
           ((o.tile_i == 1 && o.tile_j == 1) ||   // the batch kernel's pair-per-warp mode
            ((o.tile_i == 0 || o.tile_i == 32 || o.tile_i == 64) && (o.tile_j == 0 || o.tile_j == 16 || o.tile_j == 32))) &&
           std::isfinite(o.gamma0) && o.gamma0 >= 0.0 &&
           (o.gamma0 == 0.0 || (o.prune == 1 && o.reuse == 1 && std::isfinite(o.gamma_c) && o.gamma_c > 1.0));
}

// Pair-tile shape of a batch call: opts' explicit shape (mixed path), else the batch
// autotuner's table for the largest p and n; the FP64 path has 32 x 32 tiles only.
static TileShape batch_tile_shape(const lingam_opts& o, long long maxp, long long maxn) {
    if (o.precision != LINGAM_MIXED) return TileShape{32, 32};
    const TileShape t = (o.tile_i != 0 || o.tile_j != 0)
                            ? TileShape{o.tile_i ? o.tile_i : 64, o.tile_j ? o.tile_j : 32}
                            : autotune_batch_shape(maxp, maxn);
    if (t.rows == 1 && t.cols == 1 && !o.reuse) return TileShape{64, 16};   // pair mode evaluates unordered pairs
    return t;
}

// Single fits run 64 x 32, 32 x 32 or 64 x 16 tiles (32 x 16 tiles and the pair-per-warp
// mode, 1 x 1, are batch shapes).
static bool single_fit_shape(const lingam_opts& o) {
    return !(o.tile_i == 32 && o.tile_j == 16) && !(o.tile_i == 1 && o.tile_j == 1);
}

static bool is_device_ptr(const void* ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// CUDA events of the calls made by one host thread on one device: created on first need,
// reused by every later call (each call synchronises its stream before it returns, so no
// event is still pending when the next call records it), destroyed when the thread ends.
struct EventPool {
    std::vector<cudaEvent_t> ev;
    bool reserve(size_t k) {
        while (ev.size() < k) {
            cudaEvent_t e = nullptr;
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                return false;
            }
            ev.push_back(e);
        }
        return true;
    }
    ~EventPool() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        cudaGetLastError();
    }
};
static EventPool* event_pool(int dev) {
    thread_local std::map<int, EventPool> pools;
    return &pools[dev];
}

// The device view of one problem laid out in `base` (a workspace region of layout L).
// Narrow waves: waves of <= 16 columns and at least this many rows run on 128 x 16 tiles
// (LINGAM_NARROW=<rows> overrides the default; 0 turns them off, a switch for measuring them).
constexpr int kNarrowMinRows = 256;
static int narrow_min_rows() {
    static const int v = [] {
        const char* e = std::getenv("LINGAM_NARROW");
        return e && *e ? std::max(0, std::atoi(e)) : kNarrowMinRows;
    }();
    return v;
}

static Fit make_fit(char* base, const Layout& L, int p, int n, const lingam_opts& o, bool want_scores) {
    Fit f;
    std::memset(&f, 0, sizeof(f));
    f.p = p;
    f.n = n;
    f.inv_n = 1.0 / double(n);
    f.ld = L.ld;
    f.precision = o.precision;
    f.prune = o.prune;
    f.reuse = o.reuse;
    f.want_scores = want_scores ? 1 : 0;
    f.xt = base + L.off_xt;
    f.mu = reinterpret_cast<double*>(base + L.off_mu);
    f.sd = reinterpret_cast<double*>(base + L.off_sd);
    f.sig = reinterpret_cast<double*>(base + L.off_sig);
    f.sig0 = reinterpret_cast<double*>(base + L.off_sig0);
    f.sigf = reinterpret_cast<float2*>(base + L.off_sigf);
    f.hx = reinterpret_cast<double*>(base + L.off_hx);
    f.vstat = reinterpret_cast<float4*>(base + L.off_vstat);
    f.part = reinterpret_cast<double*>(base + L.off_part);
    f.cflag = reinterpret_cast<int*>(base + L.off_cflag);
    f.crow = reinterpret_cast<int*>(base + L.off_crow);
    f.prev = reinterpret_cast<double*>(base + L.off_prev);
    f.flags = reinterpret_cast<int*>(base + L.off_flags);
    f.sigma = reinterpret_cast<int*>(base + L.off_sigma);
    f.sigma_alt = reinterpret_cast<int*>(base + L.off_sigma_alt);
    f.rows = reinterpret_cast<int*>(base + L.off_rows);
    f.cols = reinterpret_cast<int*>(base + L.off_cols);
    f.order = reinterpret_cast<int*>(base + L.off_order);
    f.scratch = reinterpret_cast<int*>(base + L.off_scratch);
    f.rowsum = reinterpret_cast<double*>(base + L.off_rowsum);
    f.colsum = reinterpret_cast<double*>(base + L.off_colsum);
    f.partials = base + L.off_partials;
    f.inv_root = reinterpret_cast<double*>(base + L.off_invroot);
    f.tile_cnt = reinterpret_cast<int*>(base + L.off_tilecnt);
    f.ibuf = base + L.off_ibuf;
    f.rep_root_score = reinterpret_cast<double*>(base + L.off_rs);
    f.rep_margin = reinterpret_cast<double*>(base + L.off_rm);
    f.rep_pairs = reinterpret_cast<long long*>(base + L.off_rp);
    f.rep_scores = reinterpret_cast<double*>(base + L.off_rsc);
    f.cmat = reinterpret_cast<double*>(base + L.off_cmat);
    f.rmat = reinterpret_cast<double*>(base + L.off_rmat);
    f.rinv = reinterpret_cast<double*>(base + L.off_rinv);
    f.bout = reinterpret_cast<double*>(base + L.off_bout);
    f.ctl = reinterpret_cast<Ctl*>(base + L.off_ctl);
    f.maxtiles = L.maxtiles;
    f.maxsplit = L.maxsplit;
    f.nslots = L.nslots;
    f.split_n = o.split_n;
    f.gamma0 = o.gamma0;
    f.gamma_c = o.gamma_c;
    const TileShape ts = o.precision == LINGAM_MIXED ? choose_tile(p, n, o.tile_i, o.tile_j) : TileShape{32, 32};
    f.tile_rows = ts.rows;
    f.tile_cols = ts.cols;
    f.narrow = (o.precision == LINGAM_MIXED && ts.rows == 64 && ts.cols == 32) ? narrow_min_rows() : 0;
    return f;
}

// Prior knowledge: values in {-1, 0, 1} and no cycle among the known ancestors (prior[i][j] = 1
// is an edge j -> i); Kahn's algorithm over the p x p matrix.  Fills anc[i] = known ancestors
// of variable i.
static bool check_prior(const signed char* prior, int p, std::vector<int>& anc) {
    anc.assign(size_t(p), 0);
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j) {
            const signed char v = prior[size_t(i) * p + j];
            if (v < -1 || v > 1) return false;
            if (v == 1 && i != j) ++anc[size_t(i)];
        }
    std::vector<int> left(anc), queue;
    for (int i = 0; i < p; ++i)
        if (left[size_t(i)] == 0) queue.push_back(i);
    for (size_t q = 0; q < queue.size(); ++q) {
        const int j = queue[q];
        for (int i = 0; i < p; ++i)
            if (i != j && prior[size_t(i) * p + j] == 1 && --left[size_t(i)] == 0) queue.push_back(i);
    }
    return int(queue.size()) == p;
}

// cov_out != nullptr: stop after CalculateCovMat and copy Sigma (p x p) there.
static int fit_one(const void* X, long long p_, long long n_, int* order, double* B, void* workspace,
                   const lingam_opts& o, lingam_report* rep, double* cov_out = nullptr) {
    if (!X || !(order || cov_out) || !workspace || p_ < 1 || n_ < 3 || p_ > kMaxP || n_ > (1ll << 30) || !valid_opts(o) ||
        !single_fit_shape(o))
        return LINGAM_EINVAL;
    const int p = int(p_), n = int(n_);
    if (o.forced_order) {   // must be a permutation of 0..p-1
        std::vector<char> seen(static_cast<size_t>(p), 0);
        for (int k = 0; k < p; ++k) {
            const int v = o.forced_order[k];
            if (v < 0 || v >= p || seen[size_t(v)]) return LINGAM_EINVAL;
            seen[size_t(v)] = 1;
        }
    }
    std::vector<int> anc;
    const bool with_prior = o.prior != nullptr && !cov_out;
    if (with_prior && !check_prior(o.prior, p, anc)) return LINGAM_EINVAL;
    if (!is_device_ptr(workspace) || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0) return LINGAM_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(o.stream);
    const Layout L = make_layout(p_, n_, o.precision, o.input_dtype, with_prior);
    char* base = static_cast<char*>(workspace);
    int nsm = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LINGAM_ECUDA;

    Fit f = make_fit(base, L, p, n, o, rep && rep->scores);
    f.has_forced = o.forced_order != nullptr;
    f.forced = o.forced_order ? reinterpret_cast<const int*>(base + L.off_forced) : nullptr;
    f.prior = with_prior ? reinterpret_cast<const signed char*>(base + L.off_prior) : nullptr;
    f.anc_cnt = with_prior ? reinterpret_cast<int*>(base + L.off_anc) : nullptr;
    f.timing = o.timing ? 1 : 0;

#define CK(call)                                  \
    do {                                          \
        if ((call) != cudaSuccess) {              \
            cudaGetLastError();                   \
            return LINGAM_ECUDA;                  \
        }                                         \
    } while (0)

    Ctl c0;
    std::memset(&c0, 0, sizeof(c0));
    const double tmo = o.timeout_s > 0 ? o.timeout_s : 10.0;
    c0.timeout_ns = (unsigned long long)(tmo * 1e9);
    c0.root = -1;
    CK(cudaMemcpyAsync(f.ctl, &c0, sizeof(c0), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(f.tile_cnt, 0, size_t(L.maxtiles) * 4, st));
    if (o.forced_order)
        CK(cudaMemcpyAsync(base + L.off_forced, o.forced_order, size_t(p) * 4, cudaMemcpyHostToDevice, st));
    if (with_prior) {
        CK(cudaMemcpyAsync(base + L.off_prior, o.prior, size_t(p) * p, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(base + L.off_anc, anc.data(), size_t(p) * 4, cudaMemcpyHostToDevice, st));
    }

    const size_t in_bytes = size_t(p) * size_t(n) * (o.input_dtype == LINGAM_F32 ? 4 : 8);
    const void* xdev = X;
    if (!is_device_ptr(X)) {
        CK(cudaMemcpyAsync(base + L.off_xin, X, in_bytes, cudaMemcpyHostToDevice, st));
        xdev = base + L.off_xin;
    }

    CK(cudaMemsetAsync(f.order, 0xff, size_t(p) * 4, st));   // -1 for iterations not run
    CK(cudaMemsetAsync(f.rep_pairs, 0, size_t(p) * 8, st));
    CK(cudaMemsetAsync(f.rep_root_score, 0, size_t(p) * 8, st));
    CK(cudaMemsetAsync(f.rep_margin, 0, size_t(p) * 8, st));
    const int iters = (o.max_iters > 0 && o.max_iters < p) ? o.max_iters : p;
    const bool want_B = B != nullptr && iters == p;
    // the call's events come from this host thread's pool (created once, reused by every call)
    EventPool* pool = event_pool(dev);
    if (!pool || !pool->reserve(5 + (o.timing ? size_t(iters) + 1 : 0))) return LINGAM_ECUDA;
    const cudaEvent_t* ev = pool->ev.data();
    size_t next_ev = 5;
    std::vector<cudaEvent_t> pev;   // per-iteration pair-phase events (opts.timing)
    long long launches = 0;
    int status = LINGAM_OK;
    do {
        if (cudaEventRecord(ev[0], st) != cudaSuccess) { status = LINGAM_ECUDA; break; }
        if (inject_fault("standardize") || launch_standardize(f, xdev, o.input_dtype, st) != cudaSuccess) {
            status = LINGAM_ECUDA;
            break;
        }
        if (cudaEventRecord(ev[1], st) != cudaSuccess) { status = LINGAM_ECUDA; break; }
        if (inject_fault("covariance")) {
            status = LINGAM_ECUDA;
            break;
        }
        if (o.precision == LINGAM_MIXED) {
            if (launch_gram_tc(f, base + L.off_xin, f.partials, st) != cudaSuccess) {
                status = LINGAM_ECUDA;
                break;
            }
            launches += 4;
        } else {
            if (launch_gram(f, st) != cudaSuccess) { status = LINGAM_ECUDA; break; }
            launches += 2;
        }
        if (cudaEventRecord(ev[2], st) != cudaSuccess) { status = LINGAM_ECUDA; break; }
        if (cov_out) {
            cudaEventRecord(ev[3], st);
            cudaEventRecord(ev[4], st);
            break;
        }
        const int grid = iteration_grid(f, nsm);
        if (grid < 1) {
            status = LINGAM_ECUDA;
            break;
        }
        // opts.timing: one event before the first launch and one after each, so launch it
        // is timed between events it and it + 1 (consecutive launches share an event)
        if (o.timing) {
            const cudaEvent_t e0 = ev[next_ev++];
            pev.push_back(e0);
            cudaEventRecord(e0, st);
        }
        for (int it = 0; it < iters && status == LINGAM_OK; ++it) {
            cudaEvent_t e1 = nullptr;
            if (o.timing) {
                e1 = ev[next_ev++];
                pev.push_back(e1);
            }
            // the candidate orders alternate between the two lists: iteration it reads the
            // one the previous launch planned and plans the next into the other
            Fit fi = f;
            if (it & 1) std::swap(fi.sigma, fi.sigma_alt);
            if (inject_fault("iteration", it) || launch_iteration(fi, it, grid, st) != cudaSuccess) status = LINGAM_ECUDA;
            ++launches;
            if (o.timing) cudaEventRecord(e1, st);
        }
        if (status != LINGAM_OK) break;
        if (cudaEventRecord(ev[3], st) != cudaSuccess) { status = LINGAM_ECUDA; break; }
        if (want_B && (inject_fault("bfit") || launch_fit_B(f, st) != cudaSuccess)) { status = LINGAM_ECUDA; break; }
        if (want_B) launches += 4;
        if (cudaEventRecord(ev[4], st) != cudaSuccess) { status = LINGAM_ECUDA; break; }
    } while (0);
    if (cudaStreamSynchronize(st) != cudaSuccess) status = LINGAM_ECUDA;
    Ctl ch;
    if (status == LINGAM_OK) {
        if (cudaMemcpy(&ch, f.ctl, sizeof(ch), cudaMemcpyDeviceToHost) != cudaSuccess) status = LINGAM_ECUDA;
        else if (ch.status != 0) status = ch.status;
    }
    if (status == LINGAM_OK && cov_out) {
        if (cudaMemcpy(cov_out, f.sig, size_t(p) * p * 8, cudaMemcpyDefault) != cudaSuccess) status = LINGAM_ECUDA;
        if (rep && status == LINGAM_OK) {
            float ms = 0.f;
            rep->t_standardize_ms = cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess ? ms : -1.0;
            rep->t_gram_ms = cudaEventElapsedTime(&ms, ev[1], ev[2]) == cudaSuccess ? ms : -1.0;
            rep->kernel_launches = launches;
        }
    } else if (status == LINGAM_OK) {
        // outputs (cudaMemcpyDefault: host or device destinations)
        if (cudaMemcpyAsync(order, f.order, size_t(p) * 4, cudaMemcpyDefault, st) != cudaSuccess) status = LINGAM_ECUDA;
        if (want_B && cudaMemcpyAsync(B, f.bout, size_t(p) * p * 8, cudaMemcpyDefault, st) != cudaSuccess)
            status = LINGAM_ECUDA;
        if (rep) {
            if (rep->root_score) cudaMemcpyAsync(rep->root_score, f.rep_root_score, size_t(p) * 8, cudaMemcpyDefault, st);
            if (rep->margin_lb) cudaMemcpyAsync(rep->margin_lb, f.rep_margin, size_t(p) * 8, cudaMemcpyDefault, st);
            if (rep->pairs_evaluated)
                cudaMemcpyAsync(rep->pairs_evaluated, f.rep_pairs, size_t(p) * 8, cudaMemcpyDefault, st);
            if (rep->scores) cudaMemcpyAsync(rep->scores, f.rep_scores, size_t(p) * p * 8, cudaMemcpyDefault, st);
            float ms = 0.f;
            rep->t_standardize_ms = cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess ? ms : -1.0;
            rep->t_gram_ms = cudaEventElapsedTime(&ms, ev[1], ev[2]) == cudaSuccess ? ms : -1.0;
            rep->t_order_ms = cudaEventElapsedTime(&ms, ev[2], ev[3]) == cudaSuccess ? ms : -1.0;
            rep->t_B_ms = (want_B && cudaEventElapsedTime(&ms, ev[3], ev[4]) == cudaSuccess) ? ms : 0.0;
            double tp = 0.0;
            for (size_t k = 0; k + 1 < pev.size(); ++k)
                if (cudaEventElapsedTime(&ms, pev[k], pev[k + 1]) == cudaSuccess) {
                    tp += ms;
                    if (rep->t_pair_iter_ms && k < size_t(p)) rep->t_pair_iter_ms[k] = ms;
                }
            rep->t_pair_ms = tp;
            rep->kernel_launches = launches;
            rep->t_compute_ms = o.timing ? double(ch.phase_ns[0]) * 1e-6 : 0.0;
            rep->t_merge_ms = o.timing ? double(ch.phase_ns[1]) * 1e-6 : 0.0;
            rep->t_remove_ms = o.timing ? double(ch.phase_ns[2]) * 1e-6 : 0.0;
            rep->threshold_updates = ch.gsteps;
            rep->waves = ch.waves;
            rep->tile_pairs = ch.tile_pairs;
            rep->empty_col_pairs = ch.empty_col_pairs;
            rep->pad_row_pairs = ch.pad_row_pairs;
        }
        if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) status = LINGAM_ECUDA;
        if (rep && status == LINGAM_OK) {
            std::vector<long long> pe(static_cast<size_t>(p));
            if (cudaMemcpy(pe.data(), f.rep_pairs, size_t(p) * 8, cudaMemcpyDeviceToHost) == cudaSuccess) {
                long long tot = 0, unp = 0;
                for (int k = 0; k < iters; ++k) {
                    tot += pe[size_t(k)];
                    const long long r = p - k;
                    unp += o.reuse ? r * (r - 1) / 2 : r * (r - 1);
                }
                rep->pairs_total = tot;
                rep->pairs_unpruned = unp;
            }
        }
    }
    if (log_level() >= 1) {
        float t[4] = {-1.f, -1.f, -1.f, -1.f};
        if (status == LINGAM_OK)
            for (int k = 0; k < 4; ++k)
                if (cudaEventElapsedTime(&t[k], ev[k], ev[k + 1]) != cudaSuccess) t[k] = -1.f;
        std::fprintf(stderr,
                     "lingam: %s p=%d n=%d precision=%s status=%d (%s) launches=%lld ms: standardize %.3f covariance "
                     "%.3f order %.3f B %.3f\n",
                     cov_out ? "covariance" : "fit", p, n, o.precision == LINGAM_MIXED ? "mixed" : "fp64", status,
                     lingam_status_string(status), launches, t[0], t[1], t[2], t[3]);
    }
    cudaGetLastError();
    return status;
#undef CK
}

// ------------------------------------------------------------------ batches
// Many independent problems (uneven datasets, or bootstrap resamples of one) share
// one workspace: a header (the device Fit table, the problems' control blocks, the
// batch control block, source descriptors, row offsets, output staging, and for
// bootstraps the shared source and column indices), then one region per problem laid
// out as for a single fit.  The device work (normalisation, covariance, one
// persistent launch for all iterations of all problems, B) is captured once per
// workspace and problem shape into a CUDA graph and replayed.
struct BatchItem {
    const void* X;        // source rows (host or device)
    const int* idx;       // bootstrap: n column indices into the source row (device), else NULL
    long long ld_src;     // row stride of the source, in elements
    long long p, n;
    int* order;
    double* B;
    lingam_report* rep;
};

struct BatchLayout {
    size_t off_fits, off_ctls, off_bctl, off_src, off_rowoff, off_stage_order, off_stage_B, off_idx, off_xsrc;
    size_t header, total;
    std::vector<size_t> region;
};

static BatchLayout make_batch_layout(int count, const long long* p, const long long* n, const lingam_opts& o,
                                     size_t idx_bytes, size_t xsrc_bytes) {
    BatchLayout B;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align_up(off + bytes);
        return at;
    };
    size_t sum_p = 0, sum_pp = 0;
    for (int k = 0; k < count; ++k) {
        sum_p += size_t(p[k]);
        sum_pp += size_t(p[k]) * size_t(p[k]);
    }
    B.off_fits = take(size_t(count) * sizeof(Fit));
    B.off_ctls = take(size_t(count) * sizeof(Ctl));
    B.off_bctl = take(sizeof(Ctl));
    B.off_src = take(size_t(count) * sizeof(SrcDesc));
    B.off_rowoff = take(size_t(count + 1) * sizeof(int));
    B.off_stage_order = take(sum_p * sizeof(int));
    B.off_stage_B = take(sum_pp * sizeof(double));
    B.off_idx = take(idx_bytes);
    B.off_xsrc = take(xsrc_bytes);
    B.header = off;
    B.region.resize(size_t(count));
    for (int k = 0; k < count; ++k) B.region[size_t(k)] = take(make_layout(p[k], n[k], o.precision, o.input_dtype).total);
    B.total = off;
    return B;
}

// Copies every problem's order (and B) into the staging area, back to back.
__global__ void k_gather_outputs(const Fit* __restrict__ fits, int count, int* __restrict__ sorder,
                                 double* __restrict__ sB, int with_B) {
    const int d = blockIdx.x;
    long long po = 0, pb = 0;
    for (int e = 0; e < d; ++e) {
        po += fits[e].p;
        pb += (long long)fits[e].p * fits[e].p;
    }
    const Fit f = fits[d];
    for (int k = threadIdx.x; k < f.p; k += blockDim.x) sorder[po + k] = f.order[k];
    if (with_B)
        for (long long k = threadIdx.x; k < (long long)f.p * f.p; k += blockDim.x) sB[pb + k] = f.bout[k];
}

struct GraphKey {
    void* ws;
    int count, precision, input_dtype, prune, reuse, with_B;
    unsigned long long shape;
    bool operator<(const GraphKey& o) const {
        return std::tie(ws, count, precision, input_dtype, prune, reuse, with_B, shape) <
               std::tie(o.ws, o.count, o.precision, o.input_dtype, o.prune, o.reuse, o.with_B, o.shape);
    }
};
// Executable graphs of batch calls, by key.  At most kMaxGraphs are kept: capturing one more
// destroys the least recently launched graph that no call is using.  Keys seen once (run
// eagerly, captured on their next call) are forgotten all together past kMaxGraphSeen.
struct GraphEntry {
    cudaGraphExec_t exec;
    unsigned long long last;   // g_graph_clock at its last launch
    int busy;                  // calls between taking it and synchronising their stream
};
constexpr size_t kMaxGraphs = 32;
constexpr size_t kMaxGraphSeen = 1024;
static std::mutex g_graph_mu;
static std::map<GraphKey, GraphEntry> g_graphs;
static unsigned long long g_graph_clock = 0;
static std::map<GraphKey, int> g_graph_seen;

// Room for one more graph (caller holds g_graph_mu).
static void evict_graphs() {
    while (g_graphs.size() >= kMaxGraphs) {
        auto lru = g_graphs.end();
        for (auto it = g_graphs.begin(); it != g_graphs.end(); ++it)
            if (it->second.busy == 0 && (lru == g_graphs.end() || it->second.last < lru->second.last)) lru = it;
        if (lru == g_graphs.end()) return;   // every graph is in use: the new one is added anyway
        cudaGraphExecDestroy(lru->second.exec);
        g_graphs.erase(lru);
    }
}

// Marks a cached graph as in use for the rest of a call's scope.
struct GraphUse {
    const GraphKey* key = nullptr;
    ~GraphUse() {
        if (!key) return;
        std::lock_guard<std::mutex> lk(g_graph_mu);
        auto it = g_graphs.find(*key);
        if (it != g_graphs.end() && it->second.busy > 0) --it->second.busy;
    }
};

// Streams for the independent per-problem launches of a batch (the covariances): forked
// from the caller's stream by an event and joined back into it, so that they run
// concurrently in eager calls and become parallel branches of a captured graph.  One set
// per host thread and device, created on first use.
struct ForkStreams {
    static constexpr int kN = 8;
    cudaStream_t s[kN] = {};
    cudaEvent_t fork = nullptr, join[kN] = {};
    bool ok = false;
    void create() {
        ok = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess;
        for (int i = 0; i < kN && ok; ++i)
            ok = cudaStreamCreateWithFlags(&s[i], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) cudaGetLastError();
    }
    ~ForkStreams() {
        for (int i = 0; i < kN; ++i) {
            if (s[i]) cudaStreamDestroy(s[i]);
            if (join[i]) cudaEventDestroy(join[i]);
        }
        if (fork) cudaEventDestroy(fork);
        cudaGetLastError();
    }
};
static ForkStreams* fork_streams(int dev) {
    thread_local std::map<int, ForkStreams> sets;
    auto found = sets.find(dev);
    if (found == sets.end()) {
        found = sets.emplace(std::piecewise_construct, std::forward_as_tuple(dev), std::forward_as_tuple()).first;
        found->second.create();
    }
    return found->second.ok ? &found->second : nullptr;
}

// The device work of a batch, enqueued on st.
static cudaError_t enqueue_batch(char* ws, const BatchLayout& BL, const std::vector<Fit>& fits,
                                 const std::vector<Layout>& Ls, const lingam_opts& o, int rows, bool with_B,
                                 bool gather, int nsm, cudaStream_t st) {
    const int count = int(fits.size());
    const Fit* fits_dev = reinterpret_cast<const Fit*>(ws + BL.off_fits);
    cudaError_t e = launch_standardize_batch(fits_dev, reinterpret_cast<const SrcDesc*>(ws + BL.off_src),
                                             reinterpret_cast<const int*>(ws + BL.off_rowoff), count, rows,
                                             o.precision, o.input_dtype, st);
    if (e != cudaSuccess) return e;
    // the problems' covariances, spread over the fork streams (every stream is joined back
    // before any error returns, so a capture in progress stays well formed)
    int dev = 0;
    ForkStreams* fs = (count > 1 && cudaGetDevice(&dev) == cudaSuccess) ? fork_streams(dev) : nullptr;
    int nfork = 0;
    if (fs && cudaEventRecord(fs->fork, st) == cudaSuccess) {
        for (; nfork < ForkStreams::kN && nfork < count; ++nfork)
            if (cudaStreamWaitEvent(fs->s[nfork], fs->fork, 0) != cudaSuccess) break;
    }
    cudaGetLastError();
    // mixed path: the small problems (p <= kSmallGramP, ld <= kSmallGramLd) in one launch per
    // table chunk on the caller's stream, the others one by one on the fork streams
    const bool small_gram = o.precision == LINGAM_MIXED;
    if (small_gram) {
        std::vector<long long> ph(static_cast<size_t>(count));
        std::vector<int> lh(static_cast<size_t>(count));
        for (int k = 0; k < count; ++k) {
            ph[size_t(k)] = fits[size_t(k)].p;
            lh[size_t(k)] = fits[size_t(k)].ld;
        }
        for (int c0 = 0; c0 < count && e == cudaSuccess; c0 += kBatchLaunchMax) {
            const int cnt = std::min(kBatchLaunchMax, count - c0);
            const int units = gram_small_batch_units(ph.data() + c0, lh.data() + c0, cnt);
            if (units > 0) e = launch_gram_small_batch(fits_dev + c0, cnt, units, st);
        }
    }
    for (int k = 0, j = 0; k < count && e == cudaSuccess; ++k) {
        if (small_gram && fits[size_t(k)].p <= kSmallGramP && fits[size_t(k)].ld <= kSmallGramLd) continue;
        cudaStream_t sk = nfork > 0 ? fs->s[j++ % nfork] : st;
        e = o.precision == LINGAM_MIXED
                ? launch_gram_tc(fits[size_t(k)], ws + BL.region[size_t(k)] + Ls[size_t(k)].off_xin, fits[size_t(k)].partials, sk)
                : launch_gram(fits[size_t(k)], sk);
    }
    for (int i = 0; i < nfork; ++i) {
        const cudaError_t ej = cudaEventRecord(fs->join[i], fs->s[i]) == cudaSuccess
                                   ? cudaStreamWaitEvent(st, fs->join[i], 0)
                                   : cudaErrorUnknown;
        if (e == cudaSuccess) e = ej;
    }
    if (e != cudaSuccess) return e;
    Ctl* bctl = reinterpret_cast<Ctl*>(ws + BL.off_bctl);
    for (int c0 = 0; c0 < count; c0 += kBatchLaunchMax) {
        const int cnt = std::min(kBatchLaunchMax, count - c0);
        int maxp = 0;
        for (int k = c0; k < c0 + cnt; ++k) maxp = std::max(maxp, fits[size_t(k)].p);
        e = launch_batch(fits_dev + c0, cnt, maxp, o.precision, fits[0].tile_rows, fits[0].tile_cols, bctl, nsm, st);
        if (e != cudaSuccess) return e;
    }
    if (with_B) {
        std::vector<int> ph(static_cast<size_t>(count));
        for (int k = 0; k < count; ++k) ph[size_t(k)] = fits[size_t(k)].p;
        e = launch_fit_B_batch(fits_dev, ph.data(), count, fits.data(), st);
        if (e != cudaSuccess) return e;
    }
    if (gather) {
        k_gather_outputs<<<count, 256, 0, st>>>(fits_dev, count, reinterpret_cast<int*>(ws + BL.off_stage_order),
                                                reinterpret_cast<double*>(ws + BL.off_stage_B), with_B ? 1 : 0);
        e = cudaGetLastError();
    }
    return e;
}

// Bootstrap source shared by all problems of a batch (NULL X for plain batches).
struct BootSrc {
    const void* X;       // p x n_src rows, host or device
    const int* idx;      // nboot x n column indices, host or device
    long long p, n_src, n;
    int nboot;
};

static int fit_many(std::vector<BatchItem>& items, void* workspace, const lingam_opts& o, int* status_out,
                    const BootSrc* boot) {
    const int count = int(items.size());
    if (count == 0) return LINGAM_OK;
    if (!valid_opts(o) || o.forced_order || o.prior || o.max_iters != 0 || o.gamma0 != 0.0 || !workspace)
        return LINGAM_EINVAL;
    if (!is_device_ptr(workspace) || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0) return LINGAM_EINVAL;
    std::vector<long long> P(static_cast<size_t>(count)), N(static_cast<size_t>(count));
    bool with_B = true, gather = true;
    for (int k = 0; k < count; ++k) {
        const BatchItem& it = items[size_t(k)];
        if (!it.X || !it.order || it.p < 1 || it.n < 3 || it.p > kMaxP || it.n > (1ll << 30)) return LINGAM_EINVAL;
        P[size_t(k)] = it.p;
        N[size_t(k)] = it.n;
        if (!it.B) with_B = false;
        if (is_device_ptr(it.order) || (it.B && is_device_ptr(it.B))) gather = false;
    }
    const size_t esz = o.input_dtype == LINGAM_F32 ? 4 : 8;
    const size_t idx_bytes = boot ? size_t(boot->nboot) * size_t(boot->n) * sizeof(int) : 0;
    const size_t xsrc_bytes = boot ? size_t(boot->p) * size_t(boot->n_src) * esz : 0;
    const BatchLayout BL = make_batch_layout(count, P.data(), N.data(), o, idx_bytes, xsrc_bytes);
    char* ws = static_cast<char*>(workspace);
    cudaStream_t st = static_cast<cudaStream_t>(o.stream);
    int nsm = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LINGAM_ECUDA;
#define CKB(call)                     \
    do {                              \
        if ((call) != cudaSuccess) {  \
            cudaGetLastError();       \
            return LINGAM_ECUDA;      \
        }                             \
    } while (0)

    // bootstrap source rows and column indices (copied once into the header when on the host)
    const void* boot_x = nullptr;
    const int* boot_idx = nullptr;
    if (boot) {
        boot_x = boot->X;
        if (!is_device_ptr(boot->X)) {
            CKB(cudaMemcpyAsync(ws + BL.off_xsrc, boot->X, xsrc_bytes, cudaMemcpyHostToDevice, st));
            boot_x = ws + BL.off_xsrc;
        }
        boot_idx = boot->idx;
        if (!is_device_ptr(boot->idx)) {
            CKB(cudaMemcpyAsync(ws + BL.off_idx, boot->idx, idx_bytes, cudaMemcpyHostToDevice, st));
            boot_idx = reinterpret_cast<const int*>(ws + BL.off_idx);
        }
    }
    std::vector<char> H(BL.off_stage_order, 0);
    std::vector<Fit> fits(static_cast<size_t>(count));
    std::vector<Layout> Ls(static_cast<size_t>(count));
    Ctl c0;
    std::memset(&c0, 0, sizeof(c0));
    const double tmo = o.timeout_s > 0 ? o.timeout_s : 10.0;
    c0.timeout_ns = (unsigned long long)(tmo * 1e9);
    c0.root = -1;
    int rows = 0;
    unsigned long long shape = 1469598103934665603ull;   // FNV-1a over the problem shapes
    auto mix = [&](long long v) {
        shape ^= (unsigned long long)v;
        shape *= 1099511628211ull;
    };
    // the pair-tile shape of the whole batch: the caller's, else the batch autotuner's for the
    // largest p and n (the FP64 path: 32 x 32)
    const TileShape ts = batch_tile_shape(o, *std::max_element(P.begin(), P.end()), *std::max_element(N.begin(), N.end()));
    mix(ts.rows);
    mix(ts.cols);
    for (int k = 0; k < count; ++k) {
        BatchItem& it = items[size_t(k)];
        char* base = ws + BL.region[size_t(k)];
        Ls[size_t(k)] = make_layout(it.p, it.n, o.precision, o.input_dtype);
        const Layout& L = Ls[size_t(k)];
        Fit f = make_fit(base, L, int(it.p), int(it.n), o, it.rep && it.rep->scores);
        f.ctl = reinterpret_cast<Ctl*>(ws + BL.off_ctls) + k;
        f.tile_rows = ts.rows;
        f.tile_cols = ts.cols;
        f.narrow = 0;   // the batch kernel runs every wave on the call's tile shape
        fits[size_t(k)] = f;
        SrcDesc sd;
        if (boot) {
            sd.x = boot_x;
            sd.idx = boot_idx + size_t(k) * size_t(it.n);
            sd.ld = it.ld_src;
        } else {
            sd.x = it.X;
            if (!is_device_ptr(it.X)) {
                CKB(cudaMemcpyAsync(base + L.off_xin, it.X, size_t(it.p) * size_t(it.n) * esz, cudaMemcpyHostToDevice, st));
                sd.x = base + L.off_xin;
            }
            sd.idx = nullptr;
            sd.ld = it.n;
        }
        std::memcpy(H.data() + BL.off_fits + size_t(k) * sizeof(Fit), &f, sizeof(Fit));
        std::memcpy(H.data() + BL.off_ctls + size_t(k) * sizeof(Ctl), &c0, sizeof(Ctl));
        std::memcpy(H.data() + BL.off_src + size_t(k) * sizeof(SrcDesc), &sd, sizeof(SrcDesc));
        std::memcpy(H.data() + BL.off_rowoff + size_t(k) * sizeof(int), &rows, sizeof(int));
        rows += int(it.p);
        mix(it.p);
        mix(it.n);
        mix(it.ld_src);
        mix(it.rep && it.rep->scores ? 1 : 0);
    }
    std::memcpy(H.data() + BL.off_rowoff + size_t(count) * sizeof(int), &rows, sizeof(int));
    std::memcpy(H.data() + BL.off_bctl, &c0, sizeof(Ctl));
    // the tables at the head of the header (the staging and bootstrap areas follow them)
    CKB(cudaMemcpyAsync(ws, H.data(), BL.off_stage_order, cudaMemcpyHostToDevice, st));

    // the device work: eagerly on a key's first call (and on the legacy stream), from a
    // captured graph afterwards
    const GraphKey key{workspace, count, o.precision, o.input_dtype, o.prune, o.reuse, (with_B ? 1 : 0) | (gather ? 2 : 0) | (boot ? 4 : 0), shape};
    cudaGraphExec_t exec = nullptr;
    bool capture = false;
    GraphUse use;
    if (st != nullptr) {
        std::lock_guard<std::mutex> lk(g_graph_mu);
        auto itg = g_graphs.find(key);
        if (itg != g_graphs.end()) {
            exec = itg->second.exec;
            itg->second.last = ++g_graph_clock;
            ++itg->second.busy;
            use.key = &key;
        } else if (g_graph_seen.count(key)) {
            capture = true;
        } else {
            if (g_graph_seen.size() >= kMaxGraphSeen) g_graph_seen.clear();
            g_graph_seen[key] = 1;
        }
    }
    if (inject_fault("batch")) {
        cudaStreamSynchronize(st);   // the copies already issued finish before the call returns
        cudaGetLastError();
        return LINGAM_ECUDA;
    }
    if (exec) {
        CKB(cudaGraphLaunch(exec, st));
    } else if (capture) {
        cudaGraph_t graph = nullptr;
        bool ok = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        const cudaError_t eq = ok ? enqueue_batch(ws, BL, fits, Ls, o, rows, with_B, gather, nsm, st) : cudaErrorUnknown;
        if (ok) ok = cudaStreamEndCapture(st, &graph) == cudaSuccess && eq == cudaSuccess;
        if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        if (ok) {
            {
                std::lock_guard<std::mutex> lk(g_graph_mu);
                evict_graphs();
                auto ins = g_graphs.emplace(key, GraphEntry{exec, ++g_graph_clock, 1});
                if (!ins.second) {   // another thread captured the same key meanwhile
                    cudaGraphExecDestroy(exec);
                    exec = ins.first->second.exec;
                    ++ins.first->second.busy;
                }
                use.key = &key;
            }
            CKB(cudaGraphLaunch(exec, st));
        } else {
            CKB(enqueue_batch(ws, BL, fits, Ls, o, rows, with_B, gather, nsm, st));
        }
    } else {
        CKB(enqueue_batch(ws, BL, fits, Ls, o, rows, with_B, gather, nsm, st));
    }
    CKB(cudaStreamSynchronize(st));

    // statuses and outputs
    std::vector<Ctl> ctls(static_cast<size_t>(count));
    Ctl bc;
    CKB(cudaMemcpy(ctls.data(), ws + BL.off_ctls, size_t(count) * sizeof(Ctl), cudaMemcpyDeviceToHost));
    CKB(cudaMemcpy(&bc, ws + BL.off_bctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
    std::vector<int> sorder;
    std::vector<double> sB;
    if (gather) {
        size_t sp = 0, spp = 0;
        for (int k = 0; k < count; ++k) {
            sp += size_t(P[size_t(k)]);
            spp += size_t(P[size_t(k)]) * size_t(P[size_t(k)]);
        }
        sorder.resize(sp);
        CKB(cudaMemcpy(sorder.data(), ws + BL.off_stage_order, sp * sizeof(int), cudaMemcpyDeviceToHost));
        if (with_B) {
            sB.resize(spp);
            CKB(cudaMemcpy(sB.data(), ws + BL.off_stage_B, spp * sizeof(double), cudaMemcpyDeviceToHost));
        }
    }
    int first = LINGAM_OK;
    size_t po = 0, pb = 0;
    for (int k = 0; k < count; ++k) {
        const BatchItem& it = items[size_t(k)];
        const Fit& f = fits[size_t(k)];
        const size_t pk = size_t(it.p);
        int stk = bc.status != 0 ? bc.status : ctls[size_t(k)].status;
        if (stk == LINGAM_OK) {
            if (gather) {
                std::memcpy(it.order, sorder.data() + po, pk * sizeof(int));
                if (with_B) std::memcpy(it.B, sB.data() + pb, pk * pk * sizeof(double));
            } else {
                if (cudaMemcpy(it.order, f.order, pk * sizeof(int), cudaMemcpyDefault) != cudaSuccess) stk = LINGAM_ECUDA;
                if (with_B && cudaMemcpy(it.B, f.bout, pk * pk * sizeof(double), cudaMemcpyDefault) != cudaSuccess)
                    stk = LINGAM_ECUDA;
            }
            if (it.rep) {
                lingam_report* r = it.rep;
                if (r->root_score) cudaMemcpy(r->root_score, f.rep_root_score, pk * 8, cudaMemcpyDefault);
                if (r->margin_lb) cudaMemcpy(r->margin_lb, f.rep_margin, pk * 8, cudaMemcpyDefault);
                if (r->pairs_evaluated) cudaMemcpy(r->pairs_evaluated, f.rep_pairs, pk * 8, cudaMemcpyDefault);
                if (r->scores) cudaMemcpy(r->scores, f.rep_scores, pk * pk * 8, cudaMemcpyDefault);
                r->t_standardize_ms = r->t_gram_ms = r->t_order_ms = r->t_B_ms = r->t_pair_ms = -1.0;
                r->t_compute_ms = r->t_merge_ms = r->t_remove_ms = -1.0;
            }
        }
        po += pk;
        pb += pk * pk;
        if (status_out) status_out[k] = stk;
        if (stk != LINGAM_OK && first == LINGAM_OK) first = stk;
    }
    if (log_level() >= 1)
        std::fprintf(stderr, "lingam: batch count=%d rows=%d %s status=%d (%s) graph=%s\n", count, rows,
                     boot ? "bootstrap" : "datasets", first, lingam_status_string(first),
                     exec ? "replayed" : (capture ? "captured" : "eager"));
    cudaGetLastError();
    return first;
#undef CKB
}

}  // namespace lingam

using namespace lingam;

extern "C" {

void lingam_default_opts(lingam_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = LINGAM_MIXED;
    o->input_dtype = LINGAM_F32;
    o->prune = 1;
    o->reuse = 1;
    o->timeout_s = 10.0;
    o->gamma_c = 2.0;
}

size_t lingam_workspace_size(long long p, long long n, const lingam_opts* opts) {
    lingam_opts o;
    lingam_default_opts(&o);
    if (opts) o = *opts;
    if (p < 1 || n < 3 || p > kMaxP || n > (1ll << 30) || !valid_opts(o) || !single_fit_shape(o)) return 0;
    return make_layout(p, n, o.precision, o.input_dtype, o.prior != nullptr).total;
}

int lingam_fit(const void* X, long long p, long long n, int* order, double* B, void* workspace,
               const lingam_opts* opts, lingam_report* report) {
    lingam_opts o;
    lingam_default_opts(&o);
    if (opts) o = *opts;
    return fit_one(X, p, n, order, B, workspace, o, report);
}

int lingam_covariance(const void* X, long long p, long long n, double* Sigma, void* workspace,
                      const lingam_opts* opts, lingam_report* report) {
    lingam_opts o;
    lingam_default_opts(&o);
    if (opts) o = *opts;
    if (!Sigma || o.forced_order) return LINGAM_EINVAL;
    return fit_one(X, p, n, nullptr, nullptr, workspace, o, report, Sigma);
}

int lingam_tile_rows(long long p, long long n) {
    if (p < 1 || n < 3) return 0;
    return autotune_tile_shape(p, n).rows;
}

int lingam_tile_cols(long long p, long long n) {
    if (p < 1 || n < 3) return 0;
    return autotune_tile_shape(p, n).cols;
}

int lingam_autotune(const void* X, long long p, long long n, void* workspace, const lingam_opts* opts,
                    int* tile_rows, int* tile_cols, double* ms) {
    lingam_opts o;
    lingam_default_opts(&o);
    if (opts) o = *opts;
    if (!tile_rows || !tile_cols || o.precision != LINGAM_MIXED || o.forced_order) return LINGAM_EINVAL;
    if (p < 1 || n < 3 || p > kMaxP) return LINGAM_EINVAL;
    std::vector<int> order(static_cast<size_t>(p));
    const TileShape cand[3] = {{64, 32}, {32, 32}, {64, 16}};
    double t[3] = {0.0, 0.0, 0.0};
    int best = 0;
    for (int c = 0; c < 3; ++c) {
        lingam_opts oc = o;
        oc.tile_i = cand[c].rows;
        oc.tile_j = cand[c].cols;
        lingam_report rep;
        std::memset(&rep, 0, sizeof(rep));
        const int st = fit_one(X, p, n, order.data(), nullptr, workspace, oc, &rep);
        if (st != LINGAM_OK) return st;
        t[c] = rep.t_order_ms;
        if (t[c] < t[best]) best = c;
    }
    autotune_record(p, n, cand[best]);
    *tile_rows = cand[best].rows;
    *tile_cols = cand[best].cols;
    if (ms)
        for (int c = 0; c < 3; ++c) ms[c] = t[c];
    return LINGAM_OK;
}

void lingam_autotune_reset(void) { autotune_clear(); }

int lingam_batch_tile_rows(long long maxp, long long maxn) {
    if (maxp < 1 || maxn < 3) return 0;
    return autotune_batch_shape(maxp, maxn).rows;
}

int lingam_batch_tile_cols(long long maxp, long long maxn) {
    if (maxp < 1 || maxn < 3) return 0;
    return autotune_batch_shape(maxp, maxn).cols;
}

int lingam_autotune_batch(int count, const void* const* X, const long long* p, const long long* n, void* workspace,
                          const lingam_opts* opts, int* tile_rows, int* tile_cols, double* ms) {
    lingam_opts o;
    lingam_default_opts(&o);
    if (opts) o = *opts;
    if (count < 1 || !X || !p || !n || !workspace || !tile_rows || !tile_cols || o.precision != LINGAM_MIXED)
        return LINGAM_EINVAL;
    long long maxp = 0, maxn = 0;
    std::vector<std::vector<int>> ord(static_cast<size_t>(count));
    std::vector<int*> op(static_cast<size_t>(count));
    for (int k = 0; k < count; ++k) {
        if (p[k] < 1 || n[k] < 3 || p[k] > kMaxP) return LINGAM_EINVAL;
        maxp = std::max(maxp, p[k]);
        maxn = std::max(maxn, n[k]);
        ord[size_t(k)].resize(size_t(p[k]));
        op[size_t(k)] = ord[size_t(k)].data();
    }
    const TileShape cand[5] = {{64, 32}, {32, 32}, {64, 16}, {32, 16}, {1, 1}};
    double t[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    int best = 0;
    for (int c = 0; c < 5; ++c) {
        lingam_opts oc = o;
        oc.tile_i = cand[c].rows;
        oc.tile_j = cand[c].cols;
        // a warm-up call, the call that captures the graph, then the timed replay (three
        // eager calls on the legacy default stream); every call is synchronous
        for (int rep = 0; rep < 3; ++rep) {
            const auto t0 = std::chrono::steady_clock::now();
            const int st = lingam_fit_batch(count, X, p, n, op.data(), nullptr, workspace, &oc, nullptr, nullptr);
            const auto t1 = std::chrono::steady_clock::now();
            if (st != LINGAM_OK) return st;
            t[c] = std::chrono::duration<double, std::milli>(t1 - t0).count();
        }
        if (t[c] < t[best]) best = c;
    }
    autotune_batch_record(maxp, maxn, cand[best]);
    *tile_rows = cand[best].rows;
    *tile_cols = cand[best].cols;
    if (ms)
        for (int c = 0; c < 5; ++c) ms[c] = t[c];
    return LINGAM_OK;
}

size_t lingam_workspace_size_batch(int count, const long long* p, const long long* n, const lingam_opts* opts) {
    lingam_opts o;
    lingam_default_opts(&o);
    if (opts) o = *opts;
    if (count < 0 || (count > 0 && (!p || !n)) || !valid_opts(o)) return 0;
    for (int k = 0; k < count; ++k)
        if (p[k] < 1 || n[k] < 3 || p[k] > kMaxP || n[k] > (1ll << 30)) return 0;
    return make_batch_layout(count, p, n, o, 0, 0).total;
}

int lingam_fit_batch(int count, const void* const* X, const long long* p, const long long* n, int* const* order,
                     double* const* B, void* workspace, const lingam_opts* opts, int* status, lingam_report* report) {
    if (count < 0 || (count > 0 && (!X || !p || !n || !order || !workspace))) return LINGAM_EINVAL;
    lingam_opts o;
    lingam_default_opts(&o);
    if (opts) o = *opts;
    std::vector<BatchItem> items(static_cast<size_t>(count));
    for (int k = 0; k < count; ++k)
        items[size_t(k)] = BatchItem{X[k], nullptr, n[k], p[k], n[k], order[k], B ? B[k] : nullptr,
                                     report ? &report[k] : nullptr};
    return fit_many(items, workspace, o, status, nullptr);
}

size_t lingam_workspace_size_bootstrap(long long p, long long n, int nboot, const lingam_opts* opts) {
    lingam_opts o;
    lingam_default_opts(&o);
    if (opts) o = *opts;
    if (nboot < 1 || p < 1 || n < 3 || p > kMaxP || n > (1ll << 30) || !valid_opts(o)) return 0;
    std::vector<long long> P(static_cast<size_t>(nboot), p), N(static_cast<size_t>(nboot), n);
    const size_t esz = o.input_dtype == LINGAM_F32 ? 4 : 8;
    return make_batch_layout(nboot, P.data(), N.data(), o, size_t(nboot) * size_t(n) * sizeof(int),
                             size_t(p) * size_t(n) * esz)
        .total;
}

int lingam_fit_bootstrap(const void* X, long long p, long long n, int nboot, const int* idx, int* order, double* B,
                         void* workspace, const lingam_opts* opts, int* status, lingam_report* report) {
    if (!X || !idx || !order || !workspace || nboot < 1 || p < 1 || n < 3 || p > kMaxP || n > (1ll << 30))
        return LINGAM_EINVAL;
    lingam_opts o;
    lingam_default_opts(&o);
    if (opts) o = *opts;
    if (!is_device_ptr(idx)) {   // indices must lie in [0, n)
        for (long long k = 0; k < (long long)nboot * n; ++k)
            if (idx[k] < 0 || idx[k] >= n) return LINGAM_EINVAL;
    }
    std::vector<BatchItem> items(static_cast<size_t>(nboot));
    for (int k = 0; k < nboot; ++k)
        items[size_t(k)] = BatchItem{X, nullptr, n, p, n, order + size_t(k) * size_t(p),
                                     B ? B + size_t(k) * size_t(p) * size_t(p) : nullptr,
                                     report ? &report[k] : nullptr};
    const BootSrc boot{X, idx, p, n, n, nboot};
    return fit_many(items, workspace, o, status, &boot);
}

int lingam_selftest_wait(int which, double timeout_s, int* observed) {
    if (which < 0 || which > 3 || !(timeout_s > 0.0) || timeout_s > 60.0 || !observed) return LINGAM_EINVAL;
    int st = 0;
    if (run_wait_selftest(which, (unsigned long long)(timeout_s * 1e9), &st, nullptr) != cudaSuccess) {
        cudaGetLastError();
        return LINGAM_ECUDA;
    }
    *observed = st;
    return LINGAM_OK;
}

const char* lingam_status_string(int s) {
    switch (s) {
        case LINGAM_OK: return "ok";
        case LINGAM_EINVAL: return "invalid argument";
        case LINGAM_EDEGENERATE: return "degenerate data (zero variance, collinear pair or non-finite value)";
        case LINGAM_ENOMEM: return "out of memory";
        case LINGAM_ECUDA: return "CUDA error";
        case LINGAM_ETIMEOUT: return "device-side wait timed out";
        case LINGAM_EBOUNDS: return "index out of bounds (debug build)";
        default: return "unknown status";
    }
}

}  // extern "C"

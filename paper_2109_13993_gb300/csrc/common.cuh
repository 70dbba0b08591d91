// common.cuh -- device-side types and helpers shared by the CUDA kernels of
// the DirectLiNGAM ordering library (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "lingam.h"

namespace lingam {

// ---------------------------------------------------------------------------
// Constants of the entropy approximation, Eq. HApp (values as printed):
//   H(u) = H(nu) - k1 [E log cosh u - beta]^2 - k2 [E u exp(-u^2/2)]^2.
// H(nu) cancels in Eq. Itest, so the kernels carry H(u) - H(nu) only.
constexpr double kK1 = 79.047;
constexpr double kK2 = 7.4129;
constexpr double kBeta = 0.37457;
constexpr double kLn2 = 0.69314718055994530942;
constexpr double kLog2e = 1.44269504088896340736;

// Pair tiles: a wave has up to kTJ columns; a tile has kTI (FP64 path) or
// 2 kTI (FP32 path) rows; kPairThreads bounds the consumer threads of a CTA.
constexpr int kTI = 32;
constexpr int kTJ = 32;
constexpr int kPairThreads = 512;
// Rows of a pair tile for a precision (64 for the FP32 path, 32 for FP64).
constexpr int kChunk = 128;            // samples per shared-memory stage (FP32 path)
constexpr int kChunk64 = 64;           // samples per stage (FP64 path)
constexpr int kSub = 32;               // samples per product group (one lg2 per group)
constexpr int kStages = 3;             // TMA ring depth
constexpr int kSampleAlign = 128;      // n is padded with zero samples to a multiple of this
// A pair with 1 - rho^2 at or below this bound is degenerate (collinear to the working
// precision): on the mixed path the rows are FP32 and Sigma is exact only to about 1e-9,
// so a correlation within 2^-21 of +-1 cannot be told apart from an exact one.
__host__ __device__ constexpr double degenerate_om(bool f32) { return f32 ? 0x1p-20 : 1e-14; }
constexpr int kMaxSplit = 64;
// CTAs of a pair-kernel launch at most (two per SM of a 152-SM GB300 fit under it); the
// launches cap their grids at this bound, and the partial-moment slots of a wave (one per
// tile and CTA segment) are sized by it.
constexpr int kMaxGrid = 320;

// Flags: per variable (Fit::flags) kAlive; per candidate position (Fit::cflag) the others.
constexpr int kAlive = 1;      // still in U
constexpr int kColumned = 2;   // was a column of a wave this iteration => complete
constexpr int kDead = 4;       // partial score exceeded the best complete score
constexpr int kNoRoot = 8;     // a known ancestor is still in U (prior knowledge): never the root

// ---------------------------------------------------------------------------
// Per-fit control block in device memory.  Written by kernels, read by the
// host only after the final stream synchronisation.
struct Ctl {
    int status;          // first error (lingam_status), 0 = OK
    int it;              // current iteration
    int r;               // variables left in U at this iteration
    int root;            // root chosen at this iteration
    int done;            // iteration finished (root chosen)
    int wave;            // wave counter within the iteration
    int ncol;            // columns of the current wave
    int nrow;            // rows of the current wave (columns first, then the rest)
    int ntiles;          // row tiles of the current wave
    int pad2;
    double best;         // lowest complete score so far this iteration
    int best_var;        // variable holding `best`
    int merged;          // tiles of the current wave merged so far
    long long pairs_it;  // pairs evaluated this iteration
    unsigned long long timeout_ns;  // bound on device-side waits
    unsigned bar_count;  // grid barrier: arrivals since the fit started (never reset)
    int pad0;
    int abort;           // set when a CTA gives up a wait; the others then leave too
    int pad1;
    unsigned long long phase_ns[3];   // with timing: pair compute, merge + finalise, removal (CTA 0)
    // the next wave as published by the wave finalisation of a single fit: sequence
    // number within the iteration (bits 49-63), done (bit 48), tiles (32-47), columns
    // (24-31), rows (0-23); zero when the iteration is planned
    unsigned long long wave_word;
    // written by the iteration's last wave finalisation for the removal and the next launch:
    // U's size and the root of this iteration (the next iteration's plan, which may run
    // during this removal, overwrites r and root), and the sequence number of the last
    // published wave (wave words continue across the iterations of a fit)
    int rm_r, rm_root;
    unsigned seq0;
    int pad3;
    // the paper's threshold schedule (Fit::gamma0 > 0): the current threshold, reset to gamma0
    // at each iteration's plan, and the number of times it was raised over the fit
    double gamma;
    long long gsteps;
    // waves run over the fit, and the pairs their tiles computed (tiles x rows x columns,
    // padding and the mirrored half of the column block included)
    long long waves, tile_pairs;
    // of tile_pairs: pairs in column slots the wave left empty, and pairs of the padding rows
    // of its last tile (the rest of the waste is the duplicate half of the columns' block)
    long long empty_col_pairs, pad_row_pairs;
};

__host__ __device__ inline unsigned long long pack_wave(unsigned seq, int done, int ntiles, int ncol, int nrow) {
    return (static_cast<unsigned long long>(seq & 0x7fffu) << 49) | (static_cast<unsigned long long>(done & 1) << 48) |
           (static_cast<unsigned long long>(ntiles & 0xffff) << 32) | (static_cast<unsigned long long>(ncol & 0xff) << 24) |
           static_cast<unsigned long long>(nrow & 0xffffff);
}

// Where a batch problem's samples come from: row i of the problem is the row of
// x with stride ld (elements of the input type), sample t at column t, or at
// column idx[t] for a bootstrap resample.
struct SrcDesc {
    const void* x;
    const int* idx;
    long long ld;
};

// Device pointers of one fit, carved out of the caller's workspace.
struct Fit {
    int p;               // variables
    int n;               // samples
    double inv_n;        // 1 / n (FP64 divisions are slow on this part; the removal multiplies)
    int ld;              // padded row length (multiple of kSampleAlign)
    int precision;       // LINGAM_MIXED or LINGAM_FP64
    int prune;           // threshold pruning on
    int reuse;           // pair reuse on
    int has_forced;      // forced order given
    int want_scores;     // fill the per-iteration score matrix
    int timing;          // accumulate the phase times in Ctl::phase_ns
    void* xt;            // p x ld normalised data (float or double)
    double* mu;          // [p] row means
    double* sd;          // [p] row standard deviations (divisor n-1)
    double* sig;         // [p x p] covariance of the normalised rows, downdated each iteration
    double* sig0;        // [p x p] covariance of the normalised rows before any removal
    float2* sigf;        // [p x p] mixed path: {rho, 1 - rho^2} of sig, each formed in FP64 and
                         // rounded once: the FP32 pair kernel's coefficients without FP64 work
    double* hx;          // [p] H(x_v) - H(nu) of the current normalised rows
    float4* vstat;       // [p] per variable, for the FP32 pair path (see var_stats)
    // The current iteration's candidates are indexed by their position k in the candidate
    // list (sigma): part[k] is candidate k's partial score, its full score once complete;
    // cflag[k] holds kColumned / kDead; crow[k] is its row slot in the current wave (-1 when
    // it is not one of the wave's rows).  The plan starts them at 0, 0 and k.
    double* part;        // [p] by candidate position
    int* cflag;          // [p] by candidate position
    int* crow;           // [p] by candidate position
    double* prev;        // [p] scores of the previous iteration (ordering of candidates), by variable
    int* flags;          // [p] by variable: kAlive while the variable is in U
    int* sigma;          // [p] alive variables in candidate order
    int* sigma_alt;      // [p] the next iteration's candidate order (single fits: planned
                         // during this iteration's removal; the host swaps the two per launch)
    int* rows;           // [p] rows of the current wave (variable ids)
    int* cols;           // [kTJ] columns of the current wave
    int* order;          // [p] causal order (device copy)
    const int* forced;   // [p] forced order or nullptr
    const signed char* prior;  // [p x p] prior knowledge (prior[i p + j] = 1: x_j a known ancestor of x_i) or nullptr
    int* anc_cnt;        // [p] with prior: known ancestors of each variable still in U
    int* scratch;        // [p] wave finalisation: row slots of candidates beyond its registers;
                         // B fit: the Cholesky's row flags
    double* rowsum;      // [p] per row slot of the wave: sum over its columns of min(0, I)^2
    double* colsum;      // [maxtiles x kTJ] per tile and column: sum over the tile's rows of max(0, I)^2
    void* partials;      // [maxtiles x maxsplit x kPairThreads x 16] split partial moments (float or double)
    double* inv_root;    // [p] 1/sqrt(1 - Sigma[w,root]^2) of the current removal
    int* tile_cnt;       // [maxtiles] per-tile completion counters
    void* ibuf;          // [maxtiles x 64 x kTJ] I of the current wave's pairs (float or double)
    double* rep_root_score;  // [p]
    double* rep_margin;      // [p]
    long long* rep_pairs;    // [p]
    double* rep_scores;      // [p x p] or nullptr
    // B fit
    double* cmat;        // [p x p] covariance in causal order (original units)
    double* rmat;        // [p x p] Cholesky factor (lower)
    double* rinv;        // [p x p] inverse of the Cholesky factor
    double* bout;        // [p x p] B (original indices)
    Ctl* ctl;
    int maxtiles;        // row tiles of a wave at most (ceil(p / kTI))
    int tile_rows;       // rows of a pair tile: 64 or 32 (mixed path), 32 (FP64 path)
    int tile_cols;       // columns of a pair tile (= of a wave): 32, or 16 (mixed path)
    int maxsplit;        // sample splits at most
    int nslots;          // partial-moment slots (one per tile and CTA segment of a wave) the workspace holds
    int split_n;         // single fits: at most about split_n CTAs share a tile's samples (0 = as many as fill the grid)
    int narrow;          // single fits on 64 x 32 tiles: waves of <= 16 columns and at least this many
                         // rows run on 128 x 16 tiles (0: never)
    double gamma0;       // 0: prune against the lowest complete score; > 0: the paper's threshold
                         // schedule (Sec. III-B/C): threshold gamma0, times gamma_c while no variable
                         // can finish below it
    double gamma_c;
};

// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_status(Ctl* ctl, int code) { atomicCAS(&ctl->status, 0, code); }

// Index bound checks of the debug build (compiled with -DLINGAM_BOUNDS_CHECK): a failed check
// records LINGAM_EBOUNDS in the control block and the guarded access is skipped.  In the
// release build the checks are constant true and cost nothing.
#ifdef LINGAM_BOUNDS_CHECK
#define LINGAM_INBOUNDS(ctl, cond) ((cond) ? true : (set_status((ctl), LINGAM_EBOUNDS), false))
#else
#define LINGAM_INBOUNDS(ctl, cond) true
#endif

// The FP32 pair kernel's view of a covariance element (Fit::sigf).
__device__ __forceinline__ float2 sig_pair_f(double rho) { return make_float2(float(rho), float(fma(-rho, rho, 1.0))); }

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait until *flag becomes nonzero (the B fit's per-row readiness flags): false, with
// LINGAM_ETIMEOUT recorded in ctl, when it did not within ctl's timeout.
__device__ inline bool wait_flag_set(const volatile int* flag, Ctl* ctl) {
    unsigned long long t0 = 0, tmo = 0;
    while (*flag == 0) {
        const unsigned long long now = global_ns();
        if (t0 == 0) {
            t0 = now;
            tmo = *reinterpret_cast<volatile unsigned long long*>(&ctl->timeout_ns);
        } else if (now - t0 > tmo) {
            set_status(ctl, LINGAM_ETIMEOUT);
            return false;
        }
    }
    return true;
}

// MUFU base-2 exponential and logarithm (flush-to-zero approximations).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Sum of two float-float values (hi, lo): TwoSum of the high parts, the low parts added to
// its error, renormalised.  About 48 bits, in FP32 arithmetic.
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
    const float s = a.x + b.x, bb = s - a.x;
    const float e = (a.x - (s - bb)) + (b.x - bb) + (a.y + b.y);
    const float hi = s + e;
    return make_float2(hi, e - (hi - s));
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum (fixed shuffle tree, then fixed order over warps).
// `red` must hold blockDim.x/32 elements.  All threads get the result.
template <class T>
__device__ __forceinline__ T block_sum(T v, T* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    T s = T(0);
    for (int w = 0; w < nw; ++w) s += red[w];
    __syncthreads();
    return s;
}

// Block-wide exclusive scan of a 0/1 flag.  `red` holds blockDim.x/32 ints.
// Returns the exclusive prefix of this thread; *total gets the block total.
__device__ __forceinline__ int block_scan01(int flag, int* red, int* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    const int pre = __popc(m & ((1u << lane) - 1u));
    __syncthreads();
    if (lane == 0) red[wid] = __popc(m);
    __syncthreads();
    int off = 0, tot = 0;
    for (int w = 0; w < nw; ++w) {
        off += (w < wid) ? red[w] : 0;
        tot += red[w];
    }
    *total = tot;
    return off + pre;
}

// Adds (log cosh u - beta) and u e^{-u^2/2} of one normalised sample u (Eq. HApp)
// to a thread's running sums; FP32 on the SFU with
//   log cosh u = |u| + ln2 * log2(1 + 2^{-2 log2(e) |u|}) - ln 2,
// FP64 with the library exp and log1p.
__device__ __forceinline__ void mom_add(float u, float& lcc, float& g) {
    const float au = fabsf(u);
    const float e = ex2_approx(au * float(-2.0 * kLog2e));
    lcc += (au + float(kLn2) * lg2_approx(1.f + e)) - float(kLn2 + kBeta);
    g = fmaf(u, ex2_approx(u * u * float(-0.5 * kLog2e)), g);
}
__device__ __forceinline__ void mom_add(double u, double& lcc, double& g) {
    const double au = fabs(u);
    lcc += (au + log1p(exp(-2.0 * au))) - (kLn2 + kBeta);
    g = fma(u, exp(-0.5 * u * u), g);
}

// Entropy term of Eq. HApp minus H(nu), from the centred sums
//   lcc = sum_t (log cosh u_t - beta),  g = sum_t u_t exp(-u_t^2/2),  over n samples.
__host__ __device__ __forceinline__ double hterm(double lcc, double g, double n) {
    const double a = lcc / n, b = g / n;
    return -kK1 * a * a - kK2 * b * b;
}
__host__ __device__ __forceinline__ float hterm_f(float lcc, float g, float inv_n) {
    const float a = lcc * inv_n, b = g * inv_n;
    return -float(kK1) * a * a - float(kK2) * b * b;
}

// Statistics of one normalised row that the FP32 pair path needs, from the row's FP64
// moment sums L = sum_t (log cosh u_t - beta) and Gs = sum_t u_t exp(-u_t^2/2) over its n
// samples (row length ld with zero padding):
//   .w  the offset -kSub (ln 2 + m) of a 32-sample group, in FP32, m = mean log cosh.  The
//       pair kernel centres a residual's log-cosh group sums by its variable's own mean
//       (instead of beta), so that the FP32 sums stay small also for strongly
//       non-Gaussian variables;
//   .x  corr = (m (ld - n) - (ld / kSub) eps) / n, eps = the FP32 rounding of .w: for a
//       residual whose centred sum over the padded row is T, its mean log cosh exceeds m by
//       delta = T / n + corr exactly (padding samples have log cosh 0);
//   .y  2 (m - beta) and .z  the mean of u exp(-u^2/2), with which the entropy difference of
//       Eq. HApp between a residual and its variable is formed without the large terms:
//       H(r) - H(x) = -k1 delta (2 (m - beta) + delta) - k2 (gr - g)(gr + g).
__host__ __device__ inline float4 var_stats(double L, double Gs, int n, int ld) {
    const double m = kBeta + L / double(n);
    const double g = Gs / double(n);
    const float off = float(-double(kSub) * (kLn2 + m));
    const double eps = double(off) + double(kSub) * (kLn2 + m);
    const double corr = (m * double(ld - n) - double(ld / kSub) * eps) / double(n);
    return make_float4(float(corr), float(2.0 * (m - kBeta)), float(g), off);
}

// The same two from the removal's sums, with 1/n given (products instead of FP64 divisions,
// which are slow on this part).
__host__ __device__ __forceinline__ double hterm_inv(double lcc, double g, double inv_n) {
    const double a = lcc * inv_n, b = g * inv_n;
    return -kK1 * a * a - kK2 * b * b;
}
__host__ __device__ inline float4 var_stats_inv(double L, double Gs, int n, int ld, double inv_n) {
    const double m = kBeta + L * inv_n;
    const double g = Gs * inv_n;
    const float off = float(-double(kSub) * (kLn2 + m));
    const double eps = double(off) + double(kSub) * (kLn2 + m);
    const double corr = (m * double(ld - n) - double(ld / kSub) * eps) * inv_n;
    return make_float4(float(corr), float(2.0 * (m - kBeta)), float(g), off);
}

}  // namespace lingam

// k_iter.cu -- one iteration of the ordering loop (Algorithm 3) as one
// persistent kernel: ParaFindRoot (Algorithm 4) as a sequence of pair "waves",
// then UpdateData (Algorithm 7) and UpdateCovMat (Algorithm 8).  The grid has
// one CTA per SM and is launched cooperatively, so the phases are separated by
// grid barriers instead of kernel launches.
//
// Phases of an iteration:
//   plan     candidate order sigma of the remaining variables U, sorted by the
//            previous iteration's scores (iteration 0: H(x) - H(nu), most
//            non-Gaussian first); the first wave's columns are its first TJ.
//            Iteration 0 is planned by CTA 0 at the start of its launch; every
//            later iteration by the grid's last CTA during the previous
//            iteration's removal (into the second candidate list).
//   waves    repeat until no live candidate is left:
//     compute  every CTA evaluates its share of the wave's (tile, chunk) units
//              and writes partial sample moments;
//     merge    the tiles are spread over the CTAs; each sums its tile's partials
//              in a fixed order, evaluates I, and writes the per-row and
//              per-column score contributions; the CTA that merges the wave's
//              last tile runs the wave finalisation (scores, threshold, prune,
//              next wave or root).
//   remove   rows of U spread over the other CTAs: x_w <- (x_w - Sigma[w,root] x_root)
//            / sqrt(1 - Sigma[w,root]^2) with the new H(x_w); then the covariance
//            downdate of Eq. CovUpdate, in FP64.
//
// A wave pairs up to TJ candidate variables (the columns) with every variable
// that has not been a column yet in this iteration (the rows; the columns come
// first among the rows so that pairs inside the block are covered).  Each
// unordered pair is evaluated once and its measure I(i,j) of Eq. Itest serves
// both variables (messaging, Sec. III-A: I(j,i) = -I(i,j)).  After the wave its
// columns have met every other variable, so their scores (Algorithm 2) are
// complete; the lowest complete score bounds the root's score (threshold,
// Sec. III-B), and a variable whose partial score exceeds it can no longer be
// the root and never becomes a column.  The iteration ends when no live
// variable is left un-columned; the root is the complete variable of lowest
// score (lowest index on ties).
//
// Per pair and sample the residuals are formed from the covariance rho =
// Sigma[i,j] (Eq. var_update / Algorithm 7):
//   a = (x_i - rho x_j)/sqrt(1-rho^2) = r_i^(j),  b = (x_j - rho x_i)/sqrt(1-rho^2) = r_j^(i),
// and the two sample moments of Eq. HApp are accumulated for each:
//   sum log cosh u  with  log cosh u = |u| + ln(1 + e^{-2|u|}) - ln 2,   and sum u e^{-u^2/2}.
// The logarithm is taken once per group of kSub samples, of the product of the
// factors 1 + e^{-2|u|}; in FP32 a sample costs two SFU base-2 exponentials per
// residual.  Two consecutive samples travel together in packed f32x2
// registers.  Group sums are centred (log cosh u - beta), keeping the FP32
// running sums small.
//
// Compute work split: a wave is ntiles x (ld / CH) units (a TI x 32 pair tile
// times a chunk of CH samples).  CTA b of the G working CTAs takes units
// [b U / G, (b+1) U / G), contiguous and of equal length, and writes one
// partial slot per tile it touches (slot index tile + b is unique).  Inside a
// CTA the sample chunks of the TI + 32 variables of the current tile stream
// into a shared-memory ring with 1-D bulk copies (TMA engine) completing on
// "full" mbarriers; each warp releases a stage on its "empty" mbarrier and,
// once every warp has released it, copies its own rows of a later chunk into it.
// Every wait (mbarrier phase, grid barrier, wave word) is bounded by the fit's
// timeout.
#include <type_traits>

#include "common.cuh"
#include "launch.h"
#include "tma.cuh"

namespace lingam {

// Pair-tile shapes: TI rows x TJ columns, CONS threads of 2 x 2 pairs each (rows ty
// and ty + TI/2, columns tx and tx + 16), sample chunks of CH staged in shared-memory
// rows of LDS elements (padded: conflict-free 16-byte loads).  The FP32 path has two
// shapes, chosen by the tile autotuner: 64-row tiles of 512 threads (one CTA per SM)
// and 32-row tiles of 256 threads (two CTAs per SM, less padding waste when few
// variables remain).
template <class T_, int TI_, int TJ_, int CONS_, int CH_, int LDS_, int STAGES_, int MINB_>
struct PairShape {
    using T = T_;
    static constexpr int TI = TI_;       // tile rows
    static constexpr int TJ = TJ_;       // tile columns = columns of a wave
    static constexpr int CONS = CONS_;
    static constexpr int CH = CH_;
    static constexpr int LDS = LDS_;
    static constexpr int STAGES = STAGES_;   // copy-ring depth
    static constexpr int MINB = MINB_;   // CTAs per SM the launch bounds ask for
    static_assert(CONS == (TI / 2) * (TJ / 2), "each thread evaluates 2 x 2 pairs");
    static_assert(TJ <= kTJ, "the wave buffers hold kTJ columns");
};
using CfgF64 = PairShape<float, 64, 32, 512, kChunk, kChunk + 4, 3, 1>;      // FP32, 64 x 32 tiles
using CfgF32 = PairShape<float, 32, 32, 256, kChunk, kChunk + 4, 3, 2>;      // FP32, 32 x 32 tiles
using CfgF16 = PairShape<float, 64, 16, 256, kChunk, kChunk + 4, 2, 2>;      // FP32, 64 x 16 tiles
using CfgD = PairShape<double, 32, 32, 256, kChunk64, kChunk64 + 2, 3, 1>;   // FP64 path
// The narrow waves of the 64 x 32 kernel: a wave with 16 columns or fewer (the last wave of
// an iteration, when few candidates are left) runs on 128 x 16 tiles with the same 512
// threads and copy ring (144 rows of 64-sample chunks in each of the three stages), so its
// tiles hold the same 2048 pairs and twice the rows, instead of leaving half of the column
// slots empty.
using CfgN = PairShape<float, 128, 16, 512, kChunk / 2, kChunk / 2 + 4, 3, 1>;
constexpr int kNarrowBaseRows = CfgF64::TI;   // the tile rows of the kernel's other waves
// Batches of small problems: 32 x 16 tiles of 128 threads, 64-sample chunks, three CTAs per SM
// (a problem's late iterations, with fewer than 32 variables left, fill half the rows of a
// 64-row tile).  Batch kernel only.
using CfgB = PairShape<float, 32, 16, 128, kChunk / 2, kChunk / 2 + 4, 3, 3>;

static_assert(size_t(3) * (CfgN::TI + CfgN::TJ) * CfgN::LDS <= size_t(3) * (CfgF64::TI + CfgF64::TJ) * CfgF64::LDS,
              "the narrow waves' ring fits in the 64 x 32 kernel's");

// Rows of the tiles of a wave with ncol columns and nrow rows: narrow waves (ncol <= 16 and
// nrow >= Fit::narrow > 0) have 128-row tiles, the others tile_rows.
__host__ __device__ __forceinline__ bool wave_is_narrow(int narrow, int ncol, int nrow) {
    return narrow > 0 && ncol <= CfgN::TJ && nrow >= narrow;
}
__host__ __device__ __forceinline__ int wave_tile_rows(int narrow, int ncol, int nrow, int tile_rows) {
    return wave_is_narrow(narrow, ncol, nrow) ? CfgN::TI : tile_rows;
}

// The kernels' dynamic shared memory (copy ring, sort area, mbarriers).  Referenced by
// name in the compute loop so that its loads are shared-memory loads with 32-bit
// addresses (a generic pointer argument would make them generic loads).
extern __shared__ __align__(128) unsigned char smem_dyn[];

constexpr int kSortMax = 8192;   // candidate sort in shared memory up to this many variables
// The candidate sort's capacity of a kernel shape: the 32 x 16 batch shape keeps its shared
// memory small (three CTAs per SM), so it sorts up to 2048 candidates (larger problems keep
// index order: pruning efficiency only).
template <class Cfg>
__host__ __device__ constexpr int sort_max() {
    return std::is_same<Cfg, CfgB>::value ? 2048 : kSortMax;
}

template <class Cfg>
__host__ __device__ constexpr size_t stage_elems() {
    return size_t(Cfg::TI + Cfg::TJ) * Cfg::LDS;
}
template <class Cfg>
__host__ __device__ constexpr size_t ring_bytes() {
    return size_t(Cfg::STAGES) * stage_elems<Cfg>() * sizeof(typename Cfg::T);
}
template <class Cfg>
size_t iter_smem_bytes() {
    const size_t ring = ring_bytes<Cfg>();
    const size_t sort = size_t(sort_max<Cfg>()) * sizeof(unsigned long long);
    return (ring > sort ? ring : sort) + 2 * kStages * sizeof(uint64_t);   // full and empty barriers
}

// FP32 residuals carry the scale kScale: with u' = kScale*u,
//   e^{-u^2/2} = 2^{-u'^2},   e^{-2|u|} = 2^{kC3 |u'|}.
constexpr float kScale = 0.84932180028801904272f;     // sqrt(log2(e)/2)
constexpr float kInvScale = 1.17741002251547469101f;  // 1/kScale
constexpr float kC3 = -3.39728720115207617088f;       // -2 log2(e) / kScale

// ------------------------------------------------------------------ small helpers
// Values written by other CTAs during the same launch are read through L2 (the L1
// caches of different SMs are not coherent).
__device__ __forceinline__ int ld2(const int* p) { return __ldcg(p); }
__device__ __forceinline__ double ld2(const double* p) { return __ldcg(p); }

template <int NTH>
__device__ __forceinline__ int scan01(int flag, int* red, int* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    const int pre = __popc(m & ((1u << lane) - 1u));
    __syncthreads();
    if (lane == 0) red[wid] = __popc(m);
    __syncthreads();
    int off = 0, tot = 0;
    for (int w = 0; w < NTH / 32; ++w) {
        off += (w < wid) ? red[w] : 0;
        tot += red[w];
    }
    *total = tot;
    return off + pre;
}

// Exclusive scans of two 0/1 flags at once; red holds 2 * NTH/32 ints.
template <int NTH>
__device__ __forceinline__ void scan01x2(int fa, int fb, int* red, int* pa, int* pb, int* ta, int* tb) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned ma = __ballot_sync(0xffffffffu, fa), mb = __ballot_sync(0xffffffffu, fb);
    const unsigned below = (1u << lane) - 1u;
    __syncthreads();
    if (lane == 0) {
        red[wid] = __popc(ma);
        red[NTH / 32 + wid] = __popc(mb);
    }
    __syncthreads();
    int oa = 0, ob = 0, sa = 0, sb = 0;
    for (int w = 0; w < NTH / 32; ++w) {
        const int xa = red[w], xb = red[NTH / 32 + w];
        oa += (w < wid) ? xa : 0;
        ob += (w < wid) ? xb : 0;
        sa += xa;
        sb += xb;
    }
    *pa = oa + __popc(ma & below);
    *pb = ob + __popc(mb & below);
    *ta = sa;
    *tb = sb;
}

template <int NTH, class V>
__device__ __forceinline__ V block_sum_n(V v, V* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    V s = V(0);
    for (int w = 0; w < NTH / 32; ++w) s += red[w];
    __syncthreads();
    return s;
}

// Sum of squares in float-float arithmetic: the exact square (TwoProduct) added
// with TwoSum into a (hi, lo) pair, about 48 bits of precision on the FP32 pipe.
struct FF {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add_sq(float m) {
        const float pr = m * m, pe = fmaf(m, m, -pr);
        const float s = hi + pr, bb = s - hi;
        const float err = (hi - (s - bb)) + (pr - bb);
        hi = s;
        lo += err + pe;
    }
    __device__ __forceinline__ double value() const { return double(hi) + double(lo); }
};


// 16 consecutive values (16-byte aligned) through L2.
__device__ __forceinline__ void load16_cg(float* v, const float* src) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 x = __ldcg(reinterpret_cast<const float4*>(src) + k);
        v[4 * k + 0] = x.x;
        v[4 * k + 1] = x.y;
        v[4 * k + 2] = x.z;
        v[4 * k + 3] = x.w;
    }
}
__device__ __forceinline__ void load16_cg(double* v, const double* src) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const double2 x = __ldcg(reinterpret_cast<const double2*>(src) + k);
        v[2 * k + 0] = x.x;
        v[2 * k + 1] = x.y;
    }
}

// gpu-scope release and acquire operations for the barrier and publication protocols: a
// CTA barrier orders every thread's writes before thread 0's release, and thread 0's
// acquire before every thread's later reads.
__device__ __forceinline__ unsigned atom_add_release(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.release.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ int atom_add_acq_rel(int* p, int v) {
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" : : "l"(p), "l"(v) : "memory");
}

// Grid-wide barrier, bounded: returns false when this CTA gave up (timeout, recorded)
// or another CTA did (ctl->abort).  The arrival count only grows: it is zero when a
// fit starts and every CTA of a launch arrives once per barrier, so the arrivals at a
// barrier are those numbered [k G, (k + 1) G) for a grid of G CTAs, and a CTA waits
// until the count reaches the end of its block.  One atomic and one polling load per
// CTA; the abort flag is read by the same polls.
__device__ bool grid_sync(Ctl* ctl, unsigned long long tmo) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned G = gridDim.x;
        const unsigned old = atom_add_release(&ctl->bar_count, 1u);
        const unsigned target = old - old % G + G;
        volatile int* abortp = &ctl->abort;
        unsigned long long t0 = 0;
        for (;;) {
            const unsigned c = ld_acquire(&ctl->bar_count);
            const int ab = *abortp;
            if (ab) {
                ok = 0;
                break;
            }
            if (int(c - target) >= 0) break;
            const unsigned long long now = global_ns();
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > tmo) {
                set_status(ctl, LINGAM_ETIMEOUT);
                ctl->abort = 1;
                ok = 0;
                break;
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Bounded wait on an mbarrier phase that also gives up once the CTA (s_abort) or
// the grid (ctl->abort) has given up.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity, Ctl* ctl,
                                                   unsigned long long tmo, volatile int* s_abort) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    volatile int* abortp = &ctl->abort;
    for (;;) {
        for (int k = 0; k < 64; ++k)
            if (mbar_try_wait(bar, parity)) return true;
        if (*s_abort || *abortp) return false;
        if (global_ns() - t0 > tmo) {
            set_status(ctl, LINGAM_ETIMEOUT);
            return false;
        }
    }
}

// ------------------------------------------------------------------ unit ranges
// Working CTAs of a wave with U units on a grid of Gmax: k = ceil(U / Gmax) units
// per CTA at most, and the fewest CTAs that keep that bound, so that each tile is
// shared by as few CTAs as possible (fewer partial slots to merge, same time).
__device__ __forceinline__ long long working_ctas(long long U, long long Gmax) {
    const long long k = (U + Gmax - 1) / Gmax;
    return (U + k - 1) / k;
}
// CTA b of G owns units [lo(b), lo(b+1)), lo(b) = floor(b U / G).
__device__ __forceinline__ long long unit_lo(long long b, long long U, long long G) { return b * U / G; }
// The CTA whose range holds unit v: the smallest b with lo(b+1) > v.
__device__ __forceinline__ int cta_of_unit(long long v, long long U, long long G) {
    return int(((v + 1) * G + U - 1) / U) - 1;
}

// ------------------------------------------------------------------ plan (CTA 0)
template <int NTH, int TI, int TJ, int SORTMAX = kSortMax>
__device__ __noinline__ void plan_phase(const Fit& f, int it, unsigned char* smem, int* red, int* sigma) {
    Ctl* ctl = f.ctl;
    const int p = f.p, tid = threadIdx.x;
    int r = 0;
    for (int base = 0; base < p; base += NTH) {   // U in index order
        const int v = base + tid;
        const int a = (v < p) ? (ld2(f.flags + v) & kAlive) : 0;
        int tot;
        const int rank = r + scan01<NTH>(a ? 1 : 0, red, &tot);
        if (a && LINGAM_INBOUNDS(ctl, rank < p)) sigma[rank] = v;
        r += tot;
        __syncthreads();
    }
    // Sort by key: the order-preserving bits of the float score above the variable
    // index (ties by index).  Bitonic; compare-exchange stages with strides below 32
    // run in registers.  Beyond SORTMAX variables sigma stays in index order.
    if (r <= SORTMAX && r > 1) {
        int N = 32;
        while (N < r) N <<= 1;
        unsigned long long* key = reinterpret_cast<unsigned long long*>(smem);
        for (int k = tid; k < N; k += NTH) {
            unsigned long long kv = ~0ull;
            if (k < r) {
                const int v = sigma[k];
                const float sc = float(it == 0 ? ld2(f.hx + v) : ld2(f.prev + v));
                unsigned int bits = __float_as_uint(sc);
                bits = (bits & 0x80000000u) ? ~bits : (bits | 0x80000000u);
                kv = (static_cast<unsigned long long>(bits) << 32) | static_cast<unsigned int>(v);
            }
            key[k] = kv;
        }
        __syncthreads();
        for (int size = 2; size <= N; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                if (stride >= 32) {
                    for (int k = tid; k < N; k += NTH) {
                        const int l = k ^ stride;
                        if (l > k) {
                            const bool up = (k & size) == 0;
                            const unsigned long long a = key[k], c = key[l];
                            if ((a > c) == up) {
                                key[k] = c;
                                key[l] = a;
                            }
                        }
                    }
                    __syncthreads();
                } else {
                    for (int k0 = 0; k0 < N; k0 += NTH) {
                        const int k = k0 + tid;
                        unsigned long long a = k < N ? key[k] : ~0ull;
                        for (int st = stride; st > 0; st >>= 1) {
                            const unsigned long long c = __shfl_xor_sync(0xffffffffu, a, st);
                            const bool up = (k & size) == 0;
                            const bool lower = (k & st) == 0;
                            const unsigned long long lo = a < c ? a : c, hi = a < c ? c : a;
                            a = (lower == up) ? lo : hi;
                        }
                        if (k < N) key[k] = a;
                    }
                    __syncthreads();
                    break;
                }
            }
        }
        for (int k = tid; k < r; k += NTH) sigma[k] = int(key[k] & 0xffffffffu);
        __syncthreads();
        fence_proxy_async();   // this shared memory is the copy ring of later phases
    }
    // Prior knowledge: only variables with no known ancestor left in U can be the root; they
    // go first (a stable partition of the candidate order), the others are flagged kNoRoot
    // and take part as rows only.
    int ncand = r;
    if (f.prior && r > 1) {
        int* tmp = reinterpret_cast<int*>(smem);   // r <= kMaxP ints fit the copy ring
        for (int k = tid; k < r; k += NTH) tmp[k] = sigma[k];
        __syncthreads();
        int out = 0;
        for (int pass = 0; pass < 2; ++pass) {
            for (int base = 0; base < r; base += NTH) {
                const int k = base + tid;
                const int v = k < r ? tmp[k] : -1;
                const int c = v >= 0 && ((ld2(f.anc_cnt + v) == 0) == (pass == 0));
                int tot;
                const int rank = out + scan01<NTH>(c, red, &tot);
                if (c && LINGAM_INBOUNDS(ctl, rank < p)) sigma[rank] = v;
                out += tot;
                __syncthreads();
            }
            if (pass == 0) ncand = out;
        }
        fence_proxy_async();   // this shared memory is the copy ring of later phases
    }
    for (int k = tid; k < r; k += NTH) {   // candidate state by position; the first wave's rows
        f.part[k] = 0.0;
        f.cflag[k] = k < ncand ? 0 : kNoRoot;
        f.crow[k] = k;
        f.rows[k] = sigma[k];
    }
    if (f.want_scores)
        for (int v = tid; v < p; v += NTH) f.rep_scores[size_t(it) * p + v] = NAN;
    __syncthreads();
    if (tid == 0) {
        ctl->it = it;
        ctl->r = r;
        ctl->wave = 0;
        ctl->merged = 0;
        ctl->best = INFINITY;
        ctl->best_var = -1;
        ctl->pairs_it = 0;
        ctl->gamma = f.gamma0;
        if (r <= 1) {
            // Algorithm 2: a single remaining variable is the root
            const int root = r == 1 ? sigma[0] : -1;
            ctl->root = root;
            ctl->done = 1;
            if (root >= 0) {
                f.order[it] = root;
                if (f.want_scores) f.rep_scores[size_t(it) * p + root] = 0.0;
            }
            f.rep_root_score[it] = 0.0;
            f.rep_margin[it] = INFINITY;
            f.rep_pairs[it] = 0;
            ctl->ncol = ctl->nrow = ctl->ntiles = 0;
        } else {
            ctl->done = 0;
            const int nc = ncand < TJ ? ncand : TJ;
            for (int c = 0; c < nc; ++c) f.cols[c] = sigma[c];
            ctl->ncol = nc;
            ctl->nrow = r;
            const int ti = wave_tile_rows(f.narrow, nc, r, TI);
            ctl->ntiles = (r + ti - 1) / ti;
        }
    }
}

// Scores are sums of squares, so they are >= 0 (or +inf): their IEEE-754 bit patterns order
// like the integers they read as, and the finalisation compares them as integers instead of
// in FP64 (which runs at a small fraction of the FP32 rate on this GPU).
__device__ __forceinline__ long long okey(double x) { return __double_as_longlong(x); }

// ------------------------------------------------------------------ wave finalisation
// The wave a phase works on: its tiles, columns and rows.
struct Wave {
    int ntiles, ncol, nrow;
};

// Run by one CTA (the one that merged the wave's last tile).  The candidates' state is
// indexed by position in the candidate list, so this CTA reads it contiguously (two
// dependent round trips in all: the state, then the rows' contributions by row slot) and
// holds kPre positions per thread in registers; positions beyond kPre NTH (r > 4096 at 512
// threads) go through global memory instead.
template <int NTH, int TI, int TJ>
__device__ __noinline__ void wave_finalize(const Fit& f, const Wave& wv, int it, int* red, unsigned seq) {
    Ctl* ctl = f.ctl;
    volatile Ctl* vc = ctl;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int ncol = wv.ncol, nrow = wv.nrow, ntiles = wv.ntiles;
    const int p = f.p, r = vc->r;
    const bool reuse = f.reuse != 0;
    constexpr int NW = NTH / 32;
    constexpr int PARTS = NTH / 64;
    constexpr int SL = NTH / TJ;   // slices of the column parts
    static_assert(SL <= 32 && NW <= 32, "slices and warps fit the staging arrays");
    static_assert(TJ <= 32 && NTH >= 64, "the wave's column totals are threads 0 .. TJ - 1");
    constexpr int kPre = 8;        // candidate positions per thread held in registers
    const int nblk = (r + NTH - 1) / NTH;
    __shared__ double s_col[32 * 33];
    __shared__ double s_tot[32];
    __shared__ double s_best, s_rootpt, s_gamma;
    __shared__ int s_bestv;
    __shared__ double s_csc[32];   // the wave's complete scores, by column
    __shared__ int s_cv[32];       // and their variables

    // 1. Every load that depends on nothing written here: per candidate position k = j NTH + tid
    //    its variable, score, flags and row slot; this thread's slice of the column parts; the
    //    running threshold and pair count.
    int pv[kPre], pfl[kPre], prw[kPre];
    double ppt[kPre];
#pragma unroll
    for (int j = 0; j < kPre; ++j) {
        const int k = j * NTH + tid;
        const bool in = k < r;
        pv[j] = in ? ld2(f.sigma + k) : -1;
        ppt[j] = in ? ld2(f.part + k) : 0.0;
        pfl[j] = in ? ld2(f.cflag + k) : 0;
        prw[j] = in ? ld2(f.crow + k) : -1;
    }
    // thread (slice sl, column c) sums parts sl, sl + SL, ... of column c in that order; the
    // FP32 path's parts are float-float pairs summed in FP32 arithmetic, the FP64 path's doubles
    const int nparts = ntiles * PARTS;
    const bool ffparts = f.precision == LINGAM_MIXED;
    double ps = 0.0;
    float2 psf = make_float2(0.f, 0.f);
    {
        const int c = tid % TJ, sl = tid / TJ;
        constexpr int kB = 8;
        for (int tp = sl; tp < nparts; tp += kB * SL) {
            double v[kB];
#pragma unroll
            for (int q = 0; q < kB; ++q) {
                const int at = tp + q * SL;
                v[q] = at < nparts ? ld2(f.colsum + size_t(at) * TJ + c) : 0.0;
            }
            if (ffparts) {
#pragma unroll
                for (int q = 0; q < kB; ++q)
                    if (tp + q * SL < nparts) psf = ff_add(psf, *reinterpret_cast<const float2*>(&v[q]));
            } else {
#pragma unroll
                for (int q = 0; q < kB; ++q)
                    if (tp + q * SL < nparts) ps += v[q];
            }
        }
    }
    double best0 = INFINITY, gamma0 = 0.0;
    int bv0 = -1;
    long long pairs0 = 0;
    if (tid == 0) {
        best0 = vc->best;
        bv0 = vc->best_var;
        pairs0 = vc->pairs_it;
        gamma0 = vc->gamma;
    }
    // 2. the row contribution min(0, I(row, col))^2 summed over the wave's columns, of every
    //    candidate that is a row of this wave (by its row slot)
    double add[kPre];
#pragma unroll
    for (int j = 0; j < kPre; ++j) add[j] = (reuse && prw[j] >= 0) ? ld2(f.rowsum + prw[j]) : 0.0;
    // 3. column contributions max(0, I(row, col))^2 = min(0, I(col, row))^2: the slice sums of
    //    a column added in slice order (a fixed order)
    if (ffparts) {
        reinterpret_cast<float2*>(s_col)[(tid / TJ) * 33 + tid % TJ] = psf;
    } else {
        s_col[(tid / TJ) * 33 + tid % TJ] = ps;
    }
    __syncthreads();
    if (tid < TJ) {
        if (ffparts) {
            float2 tf = make_float2(0.f, 0.f);
            for (int j = 0; j < SL; ++j) tf = ff_add(tf, reinterpret_cast<const float2*>(s_col)[j * 33 + tid]);
            s_tot[tid] = double(tf.x) + double(tf.y);
        } else {
            double tot = 0.0;
            for (int j = 0; j < SL; ++j) tot += s_col[j * 33 + tid];
            s_tot[tid] = tot;
        }
    }
    __syncthreads();
    // 4. a column of this wave (row slot c < ncol is column c) is complete: its score so far,
    //    its own row's contribution (reuse), then its column total; the other rows add their
    //    contribution.  Lowest complete score of the wave, lowest variable index on ties.
    auto score_one = [&](int v, int e, double& pt, int& fl, double a) {
        if (e >= 0 && e < ncol) {
            const double sc = (reuse ? pt + a : pt) + s_tot[e];
            pt = sc;
            fl |= kColumned;
            if (f.want_scores) f.rep_scores[size_t(it) * p + v] = sc;
            s_csc[e] = sc;
            s_cv[e] = v;
        } else if (e >= 0 && reuse) {
            pt = pt + a;
        }
    };
#pragma unroll
    for (int j = 0; j < kPre; ++j)
        if (pv[j] >= 0) score_one(pv[j], prw[j], ppt[j], pfl[j], add[j]);
    for (int j = kPre; j < nblk; ++j) {   // positions beyond the registers
        const int k = j * NTH + tid;
        if (k >= r) continue;
        const int v = ld2(f.sigma + k), e = ld2(f.crow + k);
        double pt = ld2(f.part + k);
        int fl = ld2(f.cflag + k);
        const double a = (reuse && e >= 0) ? ld2(f.rowsum + e) : 0.0;
        score_one(v, e, pt, fl, a);
        f.part[k] = pt;
        f.cflag[k] = fl;
    }
    __syncthreads();
    if (tid < 32) {   // lowest complete score of the wave, lowest variable index on ties
        long long kc = tid < ncol ? okey(s_csc[tid]) : 0x7fffffffffffffffll;
        int vc = tid < ncol ? s_cv[tid] : 0x7fffffff;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long ko = __shfl_xor_sync(0xffffffffu, kc, o);
            const int vo = __shfl_xor_sync(0xffffffffu, vc, o);
            if (ko < kc || (ko == kc && vo < vc)) {
                kc = ko;
                vc = vo;
            }
        }
        const double sc = __longlong_as_double(kc);
        const int v = vc;
        // threshold = lowest complete score of the iteration so far
        if (tid == 0 && (bv0 < 0 || kc < okey(best0) || (kc == okey(best0) && v < bv0))) {
            best0 = sc;
            bv0 = v;
            ctl->best = sc;
            ctl->best_var = v;
        }
        if (tid == 0) {
            pairs0 += reuse ? (long long)ncol * (ncol - 1) / 2 + (long long)ncol * (nrow - ncol)
                            : (long long)ncol * (nrow - 1);
            ctl->pairs_it = pairs0;
            s_best = best0;
            s_bestv = bv0;
            s_gamma = gamma0;
        }
    }
    __syncthreads();
    const double best = s_best;
    const int bv = s_bestv;
    // the paper's threshold schedule (gamma0 > 0) in place of the running bound
    const bool gmode = f.gamma0 > 0.0 && f.prune && reuse;
    double thr = s_gamma;

    // 5. prune (partial score above the threshold), pick the next columns (the first TJ live
    //    un-columned candidates in candidate order) and rank the next rows (every other
    //    row-eligible candidate: un-columned ones with reuse, all of them without), in
    //    candidate order.  slot: a pick's column index; an eligible non-pick TJ + its rank
    //    among the non-picks (final row slot nc + rank, once nc is known); else -1.
    int slot[kPre];
    int nlive = 0, nel = 0;   // live and eligible candidates in earlier blocks
    auto rank_one = [&](int live, int elig, int& sl) {
        int pl, pe, tl, te;
        scan01x2<NTH>(live, elig, red, &pl, &pe, &tl, &te);
        const int lrank = nlive + pl;
        const bool pick = live && lrank < TJ;
        sl = pick ? lrank : (elig ? TJ + (nel + pe - min(nlive + pl, TJ)) : -1);
        nlive += tl;
        nel += te;
    };
    auto prune_one = [&](int& fl, double pt, int& live, int& elig) {
        const bool col = (fl & kColumned) != 0;
        live = 0;
        if (!col) {
            if (gmode) {   // stopped while above the current threshold; goes on once it is not
                fl = okey(pt) > okey(thr) ? (fl | kDead) : (fl & ~kDead);
            } else if (!(fl & kDead) && f.prune && reuse && okey(pt) > okey(best)) {
                fl |= kDead;
            }
            live = (fl & (kDead | kNoRoot)) ? 0 : 1;
        }
        elig = reuse ? !col : 1;
    };
    int nc = 0, nr = 0;
    for (int pass = 0;; ++pass) {
        nlive = nel = 0;
#pragma unroll
        for (int j = 0; j < kPre; ++j) {
            if (j >= nblk) break;
            int live = 0, elig = 0;
            if (pv[j] >= 0) prune_one(pfl[j], ppt[j], live, elig);
            rank_one(live, elig, slot[j]);
        }
        for (int j = kPre; j < nblk; ++j) {
            const int k = j * NTH + tid;
            int live = 0, elig = 0, sl = -1;
            if (k < r) {
                int fl = ld2(f.cflag + k);
                prune_one(fl, ld2(f.part + k), live, elig);
                f.cflag[k] = fl;
            }
            rank_one(live, elig, sl);
            if (k < r) f.scratch[k] = sl;
        }
        nc = nlive < TJ ? nlive : TJ;
        nr = nel - nc;   // every pick is eligible
        // The paper's schedule: nothing can go on and nothing finished at or below gamma (the
        // iteration cannot end yet): raise gamma by factors gamma_c until the lowest partial
        // score of a variable that may still be the root, or the lowest complete score, is at
        // or below it, and rank once more.  One raise suffices for the second pass.
        if (!gmode || nc > 0 || okey(best) <= okey(thr) || pass > 0) break;
        long long km = okey(best);
#pragma unroll
        for (int j = 0; j < kPre; ++j)
            if (pv[j] >= 0 && !(pfl[j] & (kColumned | kNoRoot))) km = min(km, okey(ppt[j]));
        for (int j = kPre; j < nblk; ++j) {
            const int k = j * NTH + tid;
            if (k < r && !(ld2(f.cflag + k) & (kColumned | kNoRoot))) km = min(km, okey(ld2(f.part + k)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) km = min(km, __shfl_xor_sync(0xffffffffu, km, o));
        if (lane == 0) s_col[wid] = __longlong_as_double(km);
        __syncthreads();
        if (tid == 0) {
            for (int w = 0; w < NW; ++w) km = min(km, okey(s_col[w]));
            const double target = __longlong_as_double(km);
            double g = thr;
            long long k = 0;
            while (g < target && k < 4096) {   // gamma_c > 1 and target finite: a few steps
                g *= f.gamma_c;
                ++k;
            }
            if (!(g >= target)) g = target;
            s_gamma = g;
            ctl->gamma = g;
            ctl->gsteps += k;
        }
        __syncthreads();
        thr = s_gamma;
    }

    // 6. the next wave's columns and rows, and the candidates' state
#pragma unroll
    for (int j = 0; j < kPre; ++j) {
        if (j >= nblk) break;
        const int k = j * NTH + tid;
        if (k < r) {
            int sl = slot[j];
            if (sl >= TJ) sl = nc + (sl - TJ);
            if (sl >= 0 && LINGAM_INBOUNDS(ctl, sl < p && (sl >= nc || sl < kTJ))) {
                f.rows[sl] = pv[j];
                if (sl < nc) f.cols[sl] = pv[j];
            }
            f.crow[k] = sl;
            f.cflag[k] = pfl[j];
            f.part[k] = ppt[j];
        }
    }
    for (int j = kPre; j < nblk; ++j) {
        const int k = j * NTH + tid;
        if (k >= r) continue;
        int sl = ld2(f.scratch + k);
        if (sl >= TJ) sl = nc + (sl - TJ);
        if (sl >= 0 && LINGAM_INBOUNDS(ctl, sl < p && (sl >= nc || sl < kTJ))) {
            const int v = ld2(f.sigma + k);
            f.rows[sl] = v;
            if (sl < nc) f.cols[sl] = v;
        }
        f.crow[k] = sl;
    }

    // 7. no live candidate left: the root is the complete variable of lowest score (or the
    //    forced one); the margin bound is the lowest other score (full if complete, else a
    //    lower bound) minus the root's; the sort keys of the next iteration's plan; and the
    //    per-row coefficients 1/sqrt(1 - Sigma[w,root]^2) of UpdateData and UpdateCovMat,
    //    computed here once for all rows in parallel.
    double second = INFINITY;
    int root = -1;
    if (nc == 0) {
        root = f.has_forced ? f.forced[it] : bv;
        const double* rootrow = f.sig + size_t(root) * p;
        const bool f32 = f.precision == LINGAM_MIXED;
        auto end_one = [&](int w, double pt, int fl) {
            if (w != bv && !(fl & kNoRoot) && okey(pt) < okey(second)) second = pt;
            f.prev[w] = pt;
            if (f.prior && f.prior[size_t(w) * p + root] == 1) f.anc_cnt[w] -= 1;   // root was a known ancestor
            if (w == root) {
                s_rootpt = pt;
                f.flags[w] = 0;
                f.inv_root[w] = 0.0;
                return;
            }
            const double c = rootrow[w];
            double om = fma(-c, c, 1.0);
            if (!(om > degenerate_om(f32))) {
                set_status(ctl, LINGAM_EDEGENERATE);
                om = 1.0;
            }
            f.inv_root[w] = rsqrt(om);
        };
#pragma unroll
        for (int j = 0; j < kPre; ++j)
            if (pv[j] >= 0) end_one(pv[j], ppt[j], pfl[j]);
        for (int j = kPre; j < nblk; ++j) {
            const int k = j * NTH + tid;
            if (k < r) end_one(ld2(f.sigma + k), ld2(f.part + k), ld2(f.cflag + k));
        }
        long long ks = okey(second);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ks = min(ks, __shfl_xor_sync(0xffffffffu, ks, o));
        if (lane == 0) s_col[wid] = __longlong_as_double(ks);
        __syncthreads();
        if (tid == 0) {
            for (int w = 0; w < NW; ++w) ks = min(ks, okey(s_col[w]));
            second = __longlong_as_double(ks);
        }
    }
    __syncthreads();   // every thread's writes precede the publication below
    if (tid == 0) {
        const int ti_next = wave_tile_rows(f.narrow, nc, nc + nr, f.narrow ? kNarrowBaseRows : TI);
        const int ntiles_next = (nc + nr + ti_next - 1) / ti_next;
        if (nc == 0) {
            ctl->root = root;
            ctl->rm_root = root;
            ctl->rm_r = r;
            if (seq != 0) ctl->seq0 = seq;
            ctl->done = 1;
            f.order[it] = root;
            f.rep_root_score[it] = root == bv ? best : s_rootpt;
            f.rep_margin[it] = second - best;
            f.rep_pairs[it] = pairs0;
        } else {
            ctl->ncol = nc;
            ctl->nrow = nc + nr;
            ctl->ntiles = ntiles_next;
        }
        ctl->merged = 0;
        if (seq != 0) {
            // publish: the CTAs of a single fit wait for this word instead of a grid barrier
            st_release64(&ctl->wave_word, pack_wave(seq, nc == 0, nc == 0 ? 0 : ntiles_next, nc, nc + nr));
        }
        // the tile counters (read by the host after the call) as atomic additions after the
        // publication, off the waves' critical path
        atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->waves), 1ull);
        atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->tile_pairs), (unsigned long long)ntiles * TI * TJ);
        atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->empty_col_pairs),
                  (unsigned long long)(TJ - ncol) * ntiles * TI);
        atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->pad_row_pairs),
                  (unsigned long long)(ntiles * TI - nrow) * ncol);
    }
}

// ------------------------------------------------------------------ per-sample math (FP32)
// Two consecutive samples of one residual u' (scaled by kScale).
struct Acc2 {
    float2 A, P, G;   // sum of |kC3 u'|, product of (1 + e^{-2|u|}), sum of u' e^{-u^2/2}; per half
};
__device__ __forceinline__ void acc2_add(Acc2& s, float2 u) {
    const float2 q = __fmul2_rn(u, u);
    float2 g;
    g.x = ex2_approx(-q.x);
    g.y = ex2_approx(-q.y);
    s.G = __ffma2_rn(u, g, s.G);
    // y = kC3 u' (kC3 < 0): e^{-2|u|} = 2^{-|y|}, the sign and the absolute value being
    // operand modifiers of the exponential
    const float2 y = __fmul2_rn(u, make_float2(kC3, kC3));
    float2 e;
    e.x = ex2_approx(-fabsf(y.x));
    e.y = ex2_approx(-fabsf(y.y));
    s.P = __ffma2_rn(s.P, e, s.P);
    s.A = __fadd2_rn(s.A, make_float2(fabsf(y.x), fabsf(y.y)));
}

// I(x_i, x_j, r_i^(j), r_j^(i)) of Eq. Itest on the FP32 path, from a pair's merged sums
// over the padded row: Ta, Tb the residuals' log-cosh sums centred by their variables'
// group offsets (var_stats .w), Ga, Gb their sums of u' exp(-u^2/2) (u' = kScale u), and
// the two variables' statistics si, sj.  Written as the difference of each residual's
// entropy (Eq. HApp) from its own variable's,
//   I = [H(r_i^(j)) - H(x_i)] - [H(r_j^(i)) - H(x_j)],
// each bracket -k1 d (2 (m - beta) + d) - k2 (g_r - g)(g_r + g) with d = T / n + corr the
// residual's mean log cosh minus its variable's, so that no FP32 term is larger than the
// difference it contributes to.
__device__ __forceinline__ float pair_measure_f(float Ta, float Ga, float Tb, float Gb, float4 si, float4 sj,
                                                float inv_n) {
    const float cg = kInvScale * inv_n;
    const float da = fmaf(Ta, inv_n, si.x), db = fmaf(Tb, inv_n, sj.x);
    const float ga = Ga * cg, gb = Gb * cg;
    const float Da = -float(kK1) * da * (si.y + da) - float(kK2) * (ga - si.z) * (ga + si.z);
    const float Db = -float(kK1) * db * (sj.y + db) - float(kK2) * (gb - sj.z) * (gb + sj.z);
    return Da - Db;
}

// Shared state of one CTA (besides the dynamic copy ring).
struct IterShared {
    int red[32];
    long long lred[33];
    int abort;
    int flag;
    double dred[32];
};

// ------------------------------------------------------------------ copy ring
// Each warp copies its share of one chunk's rows (the tile's rows, then the wave's
// columns): warp w the rows w SPW ... w SPW + SPW - 1, one 1-D bulk copy per row and
// lane.  Every row is copied (a row without a variable copies row 0 of the data, which
// no pair reads), so the stage always expects the same byte count, posted by warp 0.
// The variables of the warp's rows are kept in registers (ctile, cvar) and read again
// only when the tile changes (chunks are issued in increasing order within a wave).
template <class Cfg>
__device__ __forceinline__ void issue_part(const Fit& f, typename Cfg::T* stage, uint64_t* bar, long long unit, int nch, int nrow,
                                           int ncol, int& ctile, int& cvar) {
    using T = typename Cfg::T;
    constexpr int CH = Cfg::CH, LDS = Cfg::LDS, TI = Cfg::TI, NW = Cfg::CONS / 32;
    constexpr int TJ = Cfg::TJ;
    constexpr int SPW = (TI + TJ) / NW;
    static_assert(SPW * NW == TI + TJ && SPW <= 32, "copy rows must split evenly over the warps");
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int t = int(unit / nch), c = int(unit % nch);
    const int slot = w * SPW + lane;
    if (t != ctile) {
        ctile = t;
        int v = -1;
        if (lane < SPW) {
            if (slot < TI) {
                const int row = t * TI + slot;
                v = row < nrow ? ld2(f.rows + row) : -1;
            } else {
                v = (slot - TI) < ncol ? ld2(f.cols + slot - TI) : -1;
            }
        }
        cvar = v;
    }
    if (threadIdx.x == 0) mbar_expect_tx(bar, uint32_t(TI + TJ) * CH * sizeof(T));
    if (lane < SPW && LINGAM_INBOUNDS(f.ctl, cvar < f.p && size_t(c + 1) * CH <= size_t(f.ld))) {
        fence_proxy_async();
        const T* xt = static_cast<const T*>(f.xt);
        bulk_g2s(stage + slot * LDS, xt + size_t(cvar >= 0 ? cvar : 0) * f.ld + size_t(c) * CH, CH * sizeof(T), bar);
    }
}

// ------------------------------------------------------------------ compute phase
// Returns false when a wait gave up (the CTA then leaves the kernel).

// Where one problem's (tile, 32-sample group) units sit in the wave's stream-K
// partition: the units of all problems of the wave are concatenated, this problem's
// start at `off` of `utot`; G CTAs share them (unit_lo ranges); b_base is the first
// CTA whose range reaches this problem.  A CTA's partial slot for tile t of the
// problem is t + (b - b_base): unique within the problem, since the CTAs touching it
// are contiguous and ordered like its units.  One problem alone: {0, U, G, 0}.
struct Span {
    long long off, utot, G;
    int b_base;
};
__device__ __forceinline__ Span single_span(long long U, long long Gmax) {
    return Span{0, U, working_ctas(U, Gmax), 0};
}

template <class Cfg>
__device__ __forceinline__ bool compute_phase(const Fit& f, Ctl* gctl, const Wave& wv, const Span& sp,
                                           typename Cfg::T* ring, uint64_t* full, uint64_t* empty, IterShared& sh,
                                           int& chunk_base) {
    using T = typename Cfg::T;
    constexpr int CH = Cfg::CH, LDS = Cfg::LDS, TI = Cfg::TI, CONS = Cfg::CONS;
    constexpr bool kF32 = std::is_same<T, float>::value;
    Ctl* ctl = f.ctl;
    const int ntiles = wv.ntiles, ncol = wv.ncol, nrow = wv.nrow;
    const int p = f.p;
    // stream-K over 32-sample groups: a CTA's range of (tile, group) units may start and
    // end inside a chunk; it stages every chunk it touches, [c_lo, c_hi) in global chunk
    // index (tile * nch + chunk = group / GPC)
    constexpr int GPC = CH / kSub;
    const int nch = f.ld / CH;
    const long long ng = (long long)nch * GPC;   // groups per tile
    const long long U = (long long)ntiles * ng;
    const int b = blockIdx.x;
    if (b >= sp.G) return true;   // no unit for this CTA in this wave
    const long long g_lo = max(0ll, unit_lo(b, sp.utot, sp.G) - sp.off);
    const long long g_hi = min(U, unit_lo(b + 1, sp.utot, sp.G) - sp.off);
    if (g_lo >= g_hi) return true;   // none of this problem's units
    const int bs = b - sp.b_base;    // this CTA's partial slot offset within the problem
    const long long c_lo = g_lo / GPC;
    const int total = int((g_hi - 1) / GPC + 1 - c_lo);
    const int tid = threadIdx.x;
    const unsigned long long tmo = gctl->timeout_ns;
    const int base = chunk_base;   // ring position of this wave's first chunk

    int ctile = -1, cvar = -1;   // this thread's copy row (rows and columns changed with the wave)
    for (int k = 0; k < min(total, Cfg::STAGES); ++k) {
        const int s = (base + k) % Cfg::STAGES;
        issue_part<Cfg>(f, ring + size_t(s) * stage_elems<Cfg>(), &full[s], c_lo + k, nch, nrow, ncol, ctile, cvar);
    }
    int issued = min(total, Cfg::STAGES);   // chunks whose copies were issued

    constexpr int HJ = Cfg::TJ / 2;
    const int ty = tid / HJ, tx = tid % HJ;
    const int rsl[2] = {ty, ty + TI / 2}, csl[2] = {tx, tx + HJ};
    const T grp_off = T(-double(kSub) * (kLn2 + kBeta));
    T* parts = static_cast<T*>(f.partials);
    int k = 0;   // chunk index within this wave (this CTA)
    bool ok = true;
    for (long long u = g_lo; u < g_hi;) {
        const int t = int(u / ng);
        const long long seg_end = min(g_hi, (long long)(t + 1) * ng);   // this CTA's groups of tile t
        T s_[4], sr_[4];
        int vr[2], vc[2];   // this thread's two row and two column variables (-1: none)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int e = t * TI + rsl[h];
            vr[h] = e < nrow ? ld2(f.rows + e) : -1;
            vc[h] = csl[h] < ncol ? ld2(f.cols + csl[h]) : -1;
        }
        // FP32: the log-cosh group sums of a residual are centred by its variable's mean
        // (var_stats), the row's for r_i^(j), the column's for r_j^(i)
        float off_r[2], off_c[2];
        if constexpr (kF32) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                off_r[h] = vr[h] >= 0 ? __ldcg(&f.vstat[vr[h]].w) : float(grp_off);
                off_c[h] = vc[h] >= 0 ? __ldcg(&f.vstat[vc[h]].w) : float(grp_off);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = t * TI + rsl[q >> 1], c = csl[q & 1];
            const int vi = vr[q >> 1];
            const int vj = vc[q & 1];
            bool okp = vi >= 0 && vj >= 0;
            if (okp) okp = f.reuse ? (e >= ncol || c < e) : (vi != vj);
            if constexpr (kF32) {
                // rho and 1 - rho^2 (formed in FP64, rounded once) from the FP32 companion of Sigma
                float2 ro = okp ? __ldcg(f.sigf + size_t(vi) * p + vj) : make_float2(0.f, 1.f);
                if (okp && !(ro.y > float(degenerate_om(true)))) {
                    set_status(ctl, LINGAM_EDEGENERATE);
                    ro = make_float2(0.f, 1.f);
                }
                const float sc = kScale / sqrtf(ro.y);
                s_[q] = sc;
                sr_[q] = sc * ro.x;
            } else {
                double rho = okp ? f.sig[size_t(vi) * p + vj] : 0.0;
                double om = fma(-rho, rho, 1.0);   // 1 - rho^2 in FP64
                if (okp && !(om > degenerate_om(false))) {
                    set_status(ctl, LINGAM_EDEGENERATE);
                    om = 1.0;
                    rho = 0.0;
                }
                const double sc = 1.0 / sqrt(om);
                s_[q] = sc;
                sr_[q] = sc * rho;
            }
        }
        // D = sum over closed groups of (log cosh u - beta), Gt = sum of u e^{-u^2/2}
        T D[8], Gt[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            D[j] = T(0);
            Gt[j] = T(0);
        }
        for (long long g = u; g < seg_end; ++k) {
            const long long cg = g / GPC;   // global chunk index; k == cg - c_lo
            const int tt0 = int(g - cg * GPC) * kSub;
            const int tt1 = int(min(seg_end, (cg + 1) * GPC) - cg * GPC) * kSub;
            g = min(seg_end, (cg + 1) * GPC);
            const int pos = base + k;
            const int s = pos % Cfg::STAGES;
            const bool okw = mbar_wait_or_abort(&full[s], (pos / Cfg::STAGES) & 1, gctl, tmo, &sh.abort);
            if (!okw) sh.abort = 1;
            const T* st = reinterpret_cast<const T*>(smem_dyn) + size_t(s) * stage_elems<Cfg>();
            const T* R0 = st + rsl[0] * LDS;
            const T* R1 = st + rsl[1] * LDS;
            const T* C0 = st + (TI + csl[0]) * LDS;
            const T* C1 = st + (TI + csl[1]) * LDS;
            if (okw) {
            if constexpr (kF32) {
                float2 s2[4], sr2[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    s2[q] = make_float2(s_[q], s_[q]);
                    sr2[q] = make_float2(-sr_[q], -sr_[q]);
                }
#pragma unroll 1
                for (int tt = tt0; tt < tt1; tt += kSub) {
                    Acc2 acc[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        acc[j].A = make_float2(0.f, 0.f);
                        acc[j].P = make_float2(1.f, 1.f);
                        acc[j].G = make_float2(0.f, 0.f);
                    }
#pragma unroll 2
                    for (int uu = 0; uu < kSub; uu += 4) {
                        const float4 xr0 = *reinterpret_cast<const float4*>(R0 + tt + uu);
                        const float4 xr1 = *reinterpret_cast<const float4*>(R1 + tt + uu);
                        const float4 xc0 = *reinterpret_cast<const float4*>(C0 + tt + uu);
                        const float4 xc1 = *reinterpret_cast<const float4*>(C1 + tt + uu);
                        const float2 xi[2][2] = {{make_float2(xr0.x, xr0.y), make_float2(xr0.z, xr0.w)},
                                                 {make_float2(xr1.x, xr1.y), make_float2(xr1.z, xr1.w)}};
                        const float2 xj[2][2] = {{make_float2(xc0.x, xc0.y), make_float2(xc0.z, xc0.w)},
                                                 {make_float2(xc1.x, xc1.y), make_float2(xc1.z, xc1.w)}};
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const float2 vi = xi[q >> 1][h], vj = xj[q & 1][h];
                                const float2 a = __ffma2_rn(s2[q], vi, __fmul2_rn(sr2[q], vj));
                                const float2 bb = __ffma2_rn(s2[q], vj, __fmul2_rn(sr2[q], vi));
                                acc2_add(acc[2 * q], a);
                                acc2_add(acc[2 * q + 1], bb);
                            }
                        }
                    }
                    // close the group: one lg2 per residual for both halves' products;
                    // sum |u| = (sum |kC3 u'|) / (-kC3 kScale)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float lsum = lg2_approx(acc[j].P.x * acc[j].P.y);
                        const float asum = acc[j].A.x + acc[j].A.y;
                        const float off = (j & 1) ? off_c[(j >> 1) & 1] : off_r[j >> 2];
                        D[j] += fmaf(float(kLn2), lsum, fmaf(asum, kInvScale / -kC3, off));
                        Gt[j] += acc[j].G.x + acc[j].G.y;
                    }
                }
            } else {
#pragma unroll 1
                for (int tt = tt0; tt < tt1; tt += kSub) {
                    T A[8], P[8], Gs[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        A[j] = T(0);
                        P[j] = T(1);
                        Gs[j] = T(0);
                    }
#pragma unroll 1
                    for (int uu = 0; uu < kSub; ++uu) {
                        const double xi[2] = {R0[tt + uu], R1[tt + uu]};
                        const double xj[2] = {C0[tt + uu], C1[tt + uu]};
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const double a = fma(s_[q], xi[q >> 1], -sr_[q] * xj[q & 1]);
                            const double bb = fma(s_[q], xj[q & 1], -sr_[q] * xi[q >> 1]);
                            const double aa = fabs(a), ab = fabs(bb);
                            P[2 * q] = fma(P[2 * q], exp(-2.0 * aa), P[2 * q]);
                            P[2 * q + 1] = fma(P[2 * q + 1], exp(-2.0 * ab), P[2 * q + 1]);
                            A[2 * q] += aa;
                            A[2 * q + 1] += ab;
                            Gs[2 * q] = fma(a, exp(-0.5 * a * a), Gs[2 * q]);
                            Gs[2 * q + 1] = fma(bb, exp(-0.5 * bb * bb), Gs[2 * q + 1]);
                        }
                    }
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        D[j] += A[j] + log(P[j]) + grp_off;
                        Gt[j] += Gs[j];
                    }
                }
            }
            }
            if constexpr (Cfg::STAGES >= 3) {
                // Release without a CTA barrier: this warp arrives on the stage's empty
                // barrier; after chunk k it copies its rows of chunk k + STAGES - 1 into the
                // stage of chunk k - 1 once every warp has released that one.  Warps may
                // drift apart by up to a chunk without blocking; the copy lands while the
                // CTA computes chunk k + 1.
                if (!okw) {
                    ok = false;
                    break;
                }
                __syncwarp();
                if ((tid & 31) == 0) mbar_arrive(&empty[s]);
                const int kr = k - 1 + Cfg::STAGES;
                if (k >= 1 && kr < total) {
                    const int pr = pos - 1, sr = pr % Cfg::STAGES;
                    if (!mbar_wait_or_abort(&empty[sr], (pr / Cfg::STAGES) & 1, gctl, tmo, &sh.abort)) {
                        sh.abort = 1;
                        ok = false;
                        break;
                    }
                    issue_part<Cfg>(f, ring + size_t(sr) * stage_elems<Cfg>(), &full[sr], c_lo + kr, nch, nrow, ncol,
                                    ctile, cvar);
                    issued = kr + 1;
                }
            } else {
                // two stages: every warp is done with the stage (or a wait gave up: all leave
                // together); each warp copies its rows of the chunk STAGES further on into it
                if (__syncthreads_or(!okw)) {
                    ok = false;
                    break;
                }
                if (k + Cfg::STAGES < total) {
                    issue_part<Cfg>(f, ring + size_t(s) * stage_elems<Cfg>(), &full[s], c_lo + k + Cfg::STAGES, nch,
                                    nrow, ncol, ctile, cvar);
                    issued = k + Cfg::STAGES + 1;
                }
            }
        }
        if (__syncthreads_or(!ok)) {
            // A wait gave up (status recorded).  Give the copies still in flight a bounded
            // chance to land before the CTA leaves.
            if (tid == 0)
                for (int k2 = k; k2 < min(total, max(issued, k + Cfg::STAGES)); ++k2) {
                    const int pos = base + k2;
                    const unsigned long long t0 = global_ns();
                    while (!mbar_try_wait(&full[pos % Cfg::STAGES], (pos / Cfg::STAGES) & 1) &&
                           global_ns() - t0 < 2000000000ull) {
                    }
                }
            __syncthreads();
            return false;
        }
        // this CTA's partial moments of tile t: slot t + bs
        T* dst = parts + ((size_t(t) + bs) * CONS + tid) * 16;
        if (LINGAM_INBOUNDS(ctl, t + bs < f.nslots))
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            dst[4 * q + 0] = D[2 * q];
            dst[4 * q + 1] = Gt[2 * q];
            dst[4 * q + 2] = D[2 * q + 1];
            dst[4 * q + 3] = Gt[2 * q + 1];
        }
        u = seg_end;
    }
    chunk_base = base + total;
    return true;
}

// ------------------------------------------------------------------ merge phase
// A tile's partial slots are merged in CONS / 64 items, one per group of 64
// compute threads (256 pairs, 1024 values per slot), spread over the CTAs.  In an
// item each warp sums the slots w, w + NW, ... in order, then the warps' sums are
// added in warp order: a fixed summation order, independent of timing.  The item
// evaluates I (Eq. Itest with Eq. HApp) for its 256 pairs, which make complete
// rows of the tile: it writes those rows' contributions min(0, I)^2 over all
// columns and its part of each column's max(0, I)^2 (float-float sums, FP64
// results), and the item that completes the wave runs the wave finalisation.
template <class Cfg>
__device__ __noinline__ void merge_item(const Fit& f, const Wave& wv, const Span& sp, int it, IterShared& sh,
                                        typename Cfg::T* scratch, int item, unsigned seq) {
    using T = typename Cfg::T;
    constexpr int TI = Cfg::TI, TJ = Cfg::TJ, CONS = Cfg::CONS;
    constexpr int NW = CONS / 32;
    constexpr int PARTS = CONS / 64;            // items per tile
    constexpr bool kF32 = std::is_same<T, float>::value;
    Ctl* ctl = f.ctl;
    const int ntiles = wv.ntiles, ncol = wv.ncol, nrow = wv.nrow;
    const int ld = f.ld;
    const long long ng = ld / kSub;   // 32-sample groups per tile: the stream-K unit
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const T* parts = static_cast<const T*>(f.partials);
    const double n = double(f.n);
    const double pad_fix = double(ld - f.n) * kBeta;   // each zero padding sample added -beta
    {
        const int t = item / PARTS, part = item % PARTS;
        // slot offsets of the CTAs that hold partial moments of tile t
        const int b_first = cta_of_unit(sp.off + (long long)t * ng, sp.utot, sp.G) - sp.b_base;
        const int b_last = cta_of_unit(sp.off + (long long)(t + 1) * ng - 1, sp.utot, sp.G) - sp.b_base;
        // thread tid < 256 evaluates pair tid of the item = pair (tid & 3) of compute thread
        // part * 64 + tid / 4; its variables are fetched together with the partial moments
        const int ct = part * 64 + (tid >> 2), q = tid & 3;
        const int e_loc = ct / (TJ / 2) + (q >> 1) * (TI / 2), cc = ct % (TJ / 2) + (q & 1) * (TJ / 2);
        const int e = t * TI + e_loc;
        const int vi = (tid < 256 && e < nrow) ? ld2(f.rows + e) : -1;
        const int vj = (tid < 256 && cc < ncol) ? ld2(f.cols + cc) : -1;
        // FP32 path: the two variables' statistics, in flight while the slots are summed
        float4 si = make_float4(0.f, 0.f, 0.f, 0.f), sj = si;
        if constexpr (kF32) {
            if (vi >= 0) si = __ldcg(f.vstat + vi);
            if (vj >= 0) sj = __ldcg(f.vstat + vj);
        }
        // 1. per warp: slots b_first + wid, + NW, ...; each lane 32 of the item's 1024 values
        T acc[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) acc[k] = T(0);
        int bb = b_first + wid;
        if (!LINGAM_INBOUNDS(ctl, t + b_last < f.nslots)) bb = b_last + 1;   // no slot read
        if constexpr (kF32) {   // two slots' loads in flight; added in slot order
            for (; bb + NW <= b_last; bb += 2 * NW) {
                const T* src0 = parts + ((size_t(t) + bb) * CONS + part * 64) * 16 + lane * 32;
                const T* src1 = src0 + size_t(NW) * CONS * 16;
                T v0[32], v1[32];
                load16_cg(v0, src0);
                load16_cg(v0 + 16, src0 + 16);
                load16_cg(v1, src1);
                load16_cg(v1 + 16, src1 + 16);
#pragma unroll
                for (int k = 0; k < 32; ++k) acc[k] += v0[k];
#pragma unroll
                for (int k = 0; k < 32; ++k) acc[k] += v1[k];
            }
        }
        for (; bb <= b_last; bb += NW) {
            const T* src = parts + ((size_t(t) + bb) * CONS + part * 64) * 16 + lane * 32;
            T v[32];
            load16_cg(v, src);
            load16_cg(v + 16, src + 16);
#pragma unroll
            for (int k = 0; k < 32; ++k) acc[k] += v[k];
        }
        // warp sums to shared memory: lane-major with a pad word (conflict-free both ways)
#pragma unroll
        for (int k = 0; k < 32; ++k) scratch[wid * 1056 + lane * 33 + k] = acc[k];
        __syncthreads();
        // 2. one thread per pair: warps' sums in warp order, then I (staged past the warp sums,
        //    which other threads may still be reading)
        T* sI = scratch + NW * 1056;
        if (tid < 256) {
            T tot[4] = {T(0), T(0), T(0), T(0)};
            for (int w = 0; w < NW; ++w)
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int v = tid * 4 + k;   // value index in the item
                    tot[k] += scratch[w * 1056 + (v >> 5) * 33 + (v & 31)];
                }
            bool okp = vi >= 0 && vj >= 0;
            if (okp) okp = f.reuse ? (e >= ncol || cc < e) : (vi != vj);
            T I = T(0);
            if (okp) {
                if constexpr (kF32) {
                    I = pair_measure_f(tot[0], tot[1], tot[2], tot[3], si, sj, __frcp_rn(float(f.n)));
                } else {
                    const double ha = hterm(tot[0] + pad_fix, tot[1], n);
                    const double hb = hterm(tot[2] + pad_fix, tot[3], n);
                    I = (f.hx[vj] - f.hx[vi]) + (ha - hb);
                }
                if (!isfinite(I)) set_status(ctl, LINGAM_EDEGENERATE);
            }
            // stage the item's I: its rows are complete (all TJ columns), local row index
            // = row within the item's first half, then the second half (TI / 2 further down)
            const int el = ct / (TJ / 2) - part * (64 / (TJ / 2)) + (q >> 1) * (64 / (TJ / 2));
            sI[el * (TJ + 1) + cc] = I;
        }
        __syncthreads();
        // 3. this item's rows' contributions min(0, I)^2 over all columns (complete rows of
        //    the tile), and its part of each column's contributions max(0, I)^2; the wave's
        //    last item sums the column parts of all tiles and items in a fixed order
        constexpr int IR = 2 * (64 / (TJ / 2));   // rows of an item
        static_assert(size_t(NW) * 1056 + IR * (TJ + 1) <= ring_bytes<Cfg>() / sizeof(T),
                      "the merge scratch must fit in the copy ring");
        if (tid < IR) {
            const int e_loc = (tid < IR / 2 ? part * (IR / 2) + tid : part * (IR / 2) + tid - IR / 2 + TI / 2);
            const int e = t * TI + e_loc;
            double rs;
            if constexpr (kF32) {
                FF acc;
                for (int cc = 0; cc < TJ; ++cc) acc.add_sq(fminf(sI[tid * (TJ + 1) + cc], 0.f));
                rs = acc.value();
            } else {
                rs = 0.0;
                for (int cc = 0; cc < TJ; ++cc) {
                    const double m = fmin(double(sI[tid * (TJ + 1) + cc]), 0.0);
                    rs = fma(m, m, rs);
                }
            }
            if (e < nrow && LINGAM_INBOUNDS(ctl, e < f.p)) f.rowsum[e] = rs;
        } else if (tid >= 32 && tid < 32 + TJ) {
            const int cc = tid - 32;
            double cs;
            if constexpr (kF32) {
                FF acc;
                for (int el = 0; el < IR; ++el) acc.add_sq(fmaxf(sI[el * (TJ + 1) + cc], 0.f));
                // the column part as a float-float pair in the slot's 8 bytes
                const float2 ff = make_float2(acc.hi, acc.lo);
                cs = *reinterpret_cast<const double*>(&ff);
            } else {
                cs = 0.0;
                for (int el = 0; el < IR; ++el) {
                    const double m = fmax(double(sI[el * (TJ + 1) + cc]), 0.0);
                    cs = fma(m, m, cs);
                }
            }
            f.colsum[(size_t(t) * PARTS + part) * TJ + cc] = cs;
        }
        // the barrier orders every thread's rowsum and colsum stores before thread 0's
        // acquire-release count, which makes them visible to the CTA that counts the last
        // item (and the other items' stores to this CTA when it is that one)
        __syncthreads();
        if (tid == 0) sh.flag = (atom_add_acq_rel(&ctl->merged, 1) == ntiles * PARTS - 1);
        __syncthreads();
        if (sh.flag) wave_finalize<CONS, TI, TJ>(f, wv, it, sh.red, seq);
        __syncthreads();
    }
}

// The merge of one problem's wave: its items spread over the CTAs.
template <class Cfg>
__device__ __forceinline__ void merge_phase(const Fit& f, const Wave& wv, const Span& sp, int it, IterShared& sh,
                                            typename Cfg::T* scratch, unsigned seq) {
    const int nitems = wv.ntiles * (Cfg::CONS / 64);
    for (int item = blockIdx.x; item < nitems; item += gridDim.x)
        merge_item<Cfg>(f, wv, sp, it, sh, scratch, item, seq);
}

// ------------------------------------------------------------------ removal phases
// UpdateData (Algorithm 7) with the new H(x_w) terms; rows of U spread over the
// (virtual) CTAs, all threads of a CTA on one row.  The row coefficients
// 1/sqrt(1 - Sigma[w,root]^2) were computed by the iteration's last wave finalisation.
template <class Cfg>
__device__ __noinline__ void remove_data_phase(const Fit& f, IterShared& sh, int vb, int vG) {
    using T = typename Cfg::T;
    constexpr int NTH = Cfg::CONS;
    volatile Ctl* vc = f.ctl;
    const int r = vc->rm_r, root = vc->rm_root, p = f.p, ld = f.ld, tid = threadIdx.x;
    const int lane = tid & 31, wid = tid >> 5;
    const double* rootrow = f.sig + size_t(root) * p;
    const T* xr = static_cast<const T*>(f.xt) + size_t(root) * ld;
    for (int k = vb; k < r; k += vG) {
        const int w = ld2(f.sigma + k);
        if (w == root) continue;
        const double c = rootrow[w], inv = ld2(f.inv_root + w);
        T* xw = static_cast<T*>(f.xt) + size_t(w) * ld;
        T lcc = T(0), g = T(0);
        if constexpr (std::is_same<T, float>::value) {
            const float cc = float(c), ii = float(inv);
            float4* xw4 = reinterpret_cast<float4*>(xw);
            const float4* xr4 = reinterpret_cast<const float4*>(xr);
#pragma unroll 4
            for (int t4 = tid; t4 < ld / 4; t4 += NTH) {
                const float4 a = xw4[t4], rr = xr4[t4];
                float4 o;
                o.x = fmaf(-cc, rr.x, a.x) * ii;
                o.y = fmaf(-cc, rr.y, a.y) * ii;
                o.z = fmaf(-cc, rr.z, a.z) * ii;
                o.w = fmaf(-cc, rr.w, a.w) * ii;
                xw4[t4] = o;   // padding samples stay exactly zero
                const int t = 4 * t4;
                if (t + 0 < f.n) mom_add(o.x, lcc, g);
                if (t + 1 < f.n) mom_add(o.y, lcc, g);
                if (t + 2 < f.n) mom_add(o.z, lcc, g);
                if (t + 3 < f.n) mom_add(o.w, lcc, g);
            }
        } else {
            for (int t = tid; t < ld; t += NTH) {
                const double u = fma(-c, xr[t], xw[t]) * inv;
                xw[t] = u;
                if (t < f.n) mom_add(u, lcc, g);
            }
        }
        // per-thread sums in the working precision, warp trees, then the warp sums in FP64
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lcc += __shfl_xor_sync(0xffffffffu, lcc, o);
            g += __shfl_xor_sync(0xffffffffu, g, o);
        }
        if (lane == 0) {
            sh.dred[wid] = double(lcc);
            sh.dred[16 + wid] = double(g);
        }
        __syncthreads();
        if (tid == 0) {
            double L = 0.0, Gs = 0.0;
            for (int k2 = 0; k2 < NTH / 32; ++k2) {
                L += sh.dred[k2];
                Gs += sh.dred[16 + k2];
            }
            f.hx[w] = hterm(L, Gs, double(f.n));
            f.vstat[w] = var_stats(L, Gs, f.n, f.ld);
        }
        __syncthreads();
    }
}

// UpdateCovMat (Algorithm 8 / Eq. CovUpdate) on the normalised rows, in FP64, for
// w, j in U without the root; this CTA's rows (k = vb, vb + vG, ... of the candidate
// list) against every partner j of the list.  Sigma is symmetric, so Sigma[j,root] is
// the root's row; the root's row and column are only read, so the update is in place.
// When the list fits, the partners' indices, Sigma[root, j] and 1/sqrt(1-Sigma[root,j]^2)
// are staged in the (idle) copy ring first, so each element is one read-modify-write.
template <class Cfg>
__device__ __noinline__ void remove_cov_phase(const Fit& f, int vb, int vG) {
    constexpr int NTH = Cfg::CONS;
    volatile Ctl* vc = f.ctl;
    const int r = vc->rm_r, root = vc->rm_root, p = f.p, tid = threadIdx.x;
    const double* rootrow = f.sig + size_t(root) * p;
    const int nmine = r > vb ? (r - 1 - vb) / vG + 1 : 0;
    if (nmine == 0) return;
    const size_t stage_bytes = size_t(r) * (sizeof(int) + 2 * sizeof(double));
    if (stage_bytes <= ring_bytes<Cfg>()) {
        double* s_rj = reinterpret_cast<double*>(smem_dyn);
        double* s_ij = s_rj + r;
        int* s_j = reinterpret_cast<int*>(s_ij + r);
        for (int jj = tid; jj < r; jj += NTH) {
            const int j = ld2(f.sigma + jj);
            s_j[jj] = j;
            s_rj[jj] = rootrow[j];
            s_ij[jj] = ld2(f.inv_root + j);
        }
        __syncthreads();
        const long long total = (long long)nmine * r;
#pragma unroll 4
        for (long long idx = tid; idx < total; idx += NTH) {
            const int m = int(idx / r), jj = int(idx - (long long)m * r);
            const int kk = vb + m * vG;
            const int w = s_j[kk];
            const int j = s_j[jj];
            if (w == root || j == root) continue;
            double* row = f.sig + size_t(w) * p;
            const double nv = (j == w) ? 1.0 : (row[j] - s_rj[kk] * s_rj[jj]) * (s_ij[kk] * s_ij[jj]);
            row[j] = nv;
            if (f.precision == LINGAM_MIXED) f.sigf[size_t(w) * p + j] = sig_pair_f(nv);
        }
        __syncthreads();
        fence_proxy_async();   // the copy ring is written by bulk copies later
    } else {
        const long long total = (long long)nmine * p;
#pragma unroll 2
        for (long long idx = tid; idx < total; idx += NTH) {
            const int m = int(idx / p), j = int(idx - (long long)m * p);
            const int w = ld2(f.sigma + vb + m * vG);
            if (w == root || j == root || !(ld2(f.flags + j) & kAlive)) continue;
            double* row = f.sig + size_t(w) * p;
            const double nv =
                (j == w) ? 1.0 : (row[j] - rootrow[w] * rootrow[j]) * (ld2(f.inv_root + w) * ld2(f.inv_root + j));
            row[j] = nv;
            if (f.precision == LINGAM_MIXED) f.sigf[size_t(w) * p + j] = sig_pair_f(nv);
        }
    }
}

// UpdateData and UpdateCovMat of one CTA's rows (k = vb, vb + vG, ... of the candidate
// list) with the whole list staged in the idle copy ring first: every remaining variable's
// index, Sigma[root, j] and 1/sqrt(1 - Sigma[root, j]^2), one pass for both updates.  The
// rows stream one after another without a CTA barrier between them: each warp's sums of a
// row go to shared memory and the new H(x_w) of all rows are formed after one barrier, in
// the order of remove_data_phase (warp trees in the working precision, then the warps'
// sums in FP64 in warp order), so the results are the same.
template <class Cfg>
__host__ __device__ constexpr size_t removal_stage_bytes(int r, int nmine) {
    return size_t(r) * (sizeof(int) + 2 * sizeof(double)) + size_t(nmine) * 2 * (Cfg::CONS / 32) * sizeof(double);
}

template <class Cfg>
__device__ __noinline__ void remove_staged(const Fit& f, int vb, int vG, int r, int root, int nmine) {
    using T = typename Cfg::T;
    constexpr int NTH = Cfg::CONS, NW = NTH / 32;
    const int p = f.p, ld = f.ld, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const double* rootrow = f.sig + size_t(root) * p;
    double* s_rj = reinterpret_cast<double*>(smem_dyn);
    double* s_ij = s_rj + r;
    double* s_hp = s_ij + r;   // [nmine][2 NW]: the warps' moment sums of each row
    int* s_j = reinterpret_cast<int*>(s_hp + size_t(nmine) * 2 * NW);
    for (int jj = tid; jj < r; jj += NTH) {
        const int j = ld2(f.sigma + jj);
        s_j[jj] = j;
        s_rj[jj] = rootrow[j];
        s_ij[jj] = ld2(f.inv_root + j);
    }
    __syncthreads();
    // UpdateData (Algorithm 7) with the moments of the new rows
    const T* xr = static_cast<const T*>(f.xt) + size_t(root) * ld;
    for (int m = 0; m < nmine; ++m) {
        const int k = vb + m * vG;
        const int w = s_j[k];
        if (w == root) continue;
        const double c = s_rj[k], inv = s_ij[k];
        T* xw = static_cast<T*>(f.xt) + size_t(w) * ld;
        T lcc = T(0), g = T(0);
        if constexpr (std::is_same<T, float>::value) {
            const float cc = float(c), ii = float(inv);
            float4* xw4 = reinterpret_cast<float4*>(xw);
            const float4* xr4 = reinterpret_cast<const float4*>(xr);
            auto update4 = [&](int t4, float4 a, float4 rr) {
                float4 o;
                o.x = fmaf(-cc, rr.x, a.x) * ii;
                o.y = fmaf(-cc, rr.y, a.y) * ii;
                o.z = fmaf(-cc, rr.z, a.z) * ii;
                o.w = fmaf(-cc, rr.w, a.w) * ii;
                xw4[t4] = o;   // padding samples stay exactly zero
                const int t = 4 * t4;
                if (t + 0 < f.n) mom_add(o.x, lcc, g);
                if (t + 1 < f.n) mom_add(o.y, lcc, g);
                if (t + 2 < f.n) mom_add(o.z, lcc, g);
                if (t + 3 < f.n) mom_add(o.w, lcc, g);
            };
            const int n4 = ld / 4;
            constexpr int kPer = 8;
            if (n4 <= NTH * kPer) {
                // the thread's whole share of the row loaded first, all in flight together
                // (the stores below could alias the loads, so they would not be hoisted)
                float4 a[kPer], rr[kPer];
#pragma unroll
                for (int q = 0; q < kPer; ++q) {
                    const int t4 = tid + q * NTH;
                    if (t4 < n4) {
                        a[q] = xw4[t4];
                        rr[q] = xr4[t4];
                    }
                }
#pragma unroll
                for (int q = 0; q < kPer; ++q) {
                    const int t4 = tid + q * NTH;
                    if (t4 < n4) update4(t4, a[q], rr[q]);
                }
            } else {
#pragma unroll 4
                for (int t4 = tid; t4 < n4; t4 += NTH) update4(t4, xw4[t4], xr4[t4]);
            }
        } else {
            for (int t = tid; t < ld; t += NTH) {
                const double u = fma(-c, xr[t], xw[t]) * inv;
                xw[t] = u;
                if (t < f.n) mom_add(u, lcc, g);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lcc += __shfl_xor_sync(0xffffffffu, lcc, o);
            g += __shfl_xor_sync(0xffffffffu, g, o);
        }
        if (lane == 0) {
            s_hp[size_t(m) * 2 * NW + wid] = double(lcc);
            s_hp[size_t(m) * 2 * NW + NW + wid] = double(g);
        }
    }
    __syncthreads();
    // each row's warp sums in a warp tree, one warp per row (FP64 adds have a long latency
    // on this part, so the chains are kept short)
    const double inv_n = f.inv_n;
    for (int m = wid; m < nmine; m += NW) {
        const int w = s_j[vb + m * vG];
        if (w == root) continue;
        double L = lane < NW ? s_hp[size_t(m) * 2 * NW + lane] : 0.0;
        double Gs = lane < NW ? s_hp[size_t(m) * 2 * NW + NW + lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            L += __shfl_xor_sync(0xffffffffu, L, o);
            Gs += __shfl_xor_sync(0xffffffffu, Gs, o);
        }
        if (lane == 0) {
            f.hx[w] = hterm_inv(L, Gs, inv_n);
            f.vstat[w] = var_stats_inv(L, Gs, f.n, f.ld, inv_n);
        }
    }
    // UpdateCovMat (Algorithm 8 / Eq. CovUpdate), FP64.  Sigma stays symmetric, so each
    // unordered pair of U is updated once, by the CTA holding the row of its lower candidate
    // position, which writes both of its elements (and both of the FP32 view's); a CTA reads
    // only elements it writes itself.  Half the FP64 work of a full update, which the FP64
    // rate of this part bounds.
    for (int m = 0; m < nmine; ++m) {
        const int kk = vb + m * vG;
        const int w = s_j[kk];
        if (w == root) continue;
        const double aw = s_rj[kk], bw = s_ij[kk];
        double* row = f.sig + size_t(w) * p;
        if (tid == 0) {
            row[w] = 1.0;
            if constexpr (std::is_same<T, float>::value) f.sigf[size_t(w) * p + w] = sig_pair_f(1.0);
        }
        for (int jj = kk + 1 + tid; jj < r; jj += NTH) {
            const int j = s_j[jj];
            if (j == root) continue;
            const double nv = (row[j] - aw * s_rj[jj]) * (bw * s_ij[jj]);
            row[j] = nv;
            f.sig[size_t(j) * p + w] = nv;
            if constexpr (std::is_same<T, float>::value) {
                const float2 fv = sig_pair_f(nv);
                f.sigf[size_t(w) * p + j] = fv;
                f.sigf[size_t(j) * p + w] = fv;
            }
        }
    }
    __syncthreads();
    fence_proxy_async();   // the copy ring is written by bulk copies later
}

// ------------------------------------------------------------------ the iteration kernel
// The end of an iteration that took a root.  The grid's last CTA plans the next iteration
// (its candidate order into f.sigma_alt, which the host passes as f.sigma to the next
// launch): the plan needs the scores and U without the root, not the removal's results.
// The other CTAs remove the root: UpdateData and UpdateCovMat touch disjoint memory (the
// covariance's root column, from which the coefficients come, is not written) and none of
// what the plan writes.  Out of line, so that the kernel around the pair waves stays small.
template <class Cfg>
__device__ __noinline__ void iteration_tail(const Fit& f, int it, IterShared& sh) {
    if (*reinterpret_cast<volatile int*>(&f.ctl->rm_root) < 0) return;
    const int fc = int(gridDim.x) - 1;
    if (int(blockIdx.x) == fc) {
        plan_phase<Cfg::CONS, Cfg::TI, Cfg::TJ>(f, it + 1, smem_dyn, sh.red, f.sigma_alt);
    } else {
        volatile Ctl* vc = f.ctl;
        const int r = vc->rm_r, root = vc->rm_root, vb = int(blockIdx.x), vG = int(gridDim.x) - 1;
        if (r <= vb) return;   // no row of U for this CTA
        const int nmine = (r - 1 - vb) / vG + 1;
        if (removal_stage_bytes<Cfg>(r, nmine) <= ring_bytes<Cfg>()) {
            remove_staged<Cfg>(f, vb, vG, r, root, nmine);
        } else {
            remove_data_phase<Cfg>(f, sh, vb, vG);
            remove_cov_phase<Cfg>(f, vb, vG);
        }
    }
}

// A narrow wave's compute phase, grid barrier and merge, out of line: the 64 x 32 kernel's
// own sample loop stays the only one inlined into it (its speed depends on that).  Returns
// false when the CTA must leave the kernel.
template <class Cfg>
__device__ __noinline__ bool narrow_wave(const Fit& f, Ctl* ctl, const Wave& wv, const Span& sp,
                                         typename Cfg::T* ring, uint64_t* full, uint64_t* empty, IterShared& sh,
                                         int& chunk_base, int it, unsigned seq, unsigned long long tmo, bool timed,
                                         unsigned long long& tph) {
    if (!compute_phase<Cfg>(f, ctl, wv, sp, ring, full, empty, sh, chunk_base)) {
        ctl->abort = 1;
        return false;
    }
    if (!grid_sync(ctl, tmo)) return false;
    if (timed) {
        const unsigned long long t = global_ns();
        ctl->phase_ns[0] += t - tph;
        tph = t;
    }
    merge_phase<Cfg>(f, wv, sp, it, sh, ring, seq);
    return true;
}

// Wait (bounded) until the wave finalisation of a single fit has published wave word
// seq; returns the next wave and whether the iteration is done.  Returns false when
// this CTA gave up (timeout, recorded) or another CTA did.
__device__ bool wait_wave(Ctl* ctl, unsigned seq, unsigned long long tmo, Wave& wv, bool& done) {
    __shared__ unsigned long long s_word;
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile int* abortp = &ctl->abort;
        unsigned long long w = 0, t0 = 0;
        for (;;) {
            w = ld_acquire64(&ctl->wave_word);
            const int ab = *abortp;
            if (ab) {
                ok = 0;
                break;
            }
            if (unsigned(w >> 49) == (seq & 0x7fffu)) break;
            const unsigned long long now = global_ns();
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > tmo) {
                set_status(ctl, LINGAM_ETIMEOUT);
                ctl->abort = 1;
                ok = 0;
                break;
            }
        }
        s_word = w;
        s_ok = ok;
    }
    __syncthreads();
    const unsigned long long w = s_word;
    const int ok = s_ok;
    __syncthreads();   // s_word and s_ok are reused by the next wait
    done = ((w >> 48) & 1) != 0;
    wv.ntiles = int((w >> 32) & 0xffff);
    wv.ncol = int((w >> 24) & 0xff);
    wv.nrow = int(w & 0xffffff);
    return ok != 0;
}

template <class Cfg>
__global__ void __launch_bounds__(Cfg::CONS, Cfg::MINB) k_iteration(Fit f, int it) {
    unsigned char* smem_raw = smem_dyn;
    __shared__ IterShared sh;
    using T = typename Cfg::T;
    Ctl* ctl = f.ctl;
    T* ring = reinterpret_cast<T*>(smem_raw);
    const size_t ring_or_sort = ring_bytes<Cfg>() > size_t(kSortMax) * 8 ? ring_bytes<Cfg>() : size_t(kSortMax) * 8;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + ring_or_sort);
    uint64_t* empty = full + kStages;
    volatile Ctl* vc = ctl;
    // A failure recorded before this launch: every CTA reads it before the first
    // barrier, so all of them leave together.
    if (vc->status != 0) return;
    const unsigned long long tmo = vc->timeout_ns;
    if (threadIdx.x == 0) {
        for (int s = 0; s < Cfg::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], Cfg::CONS / 32);
        }
        sh.abort = 0;
        fence_barrier_init();
    }
    __syncthreads();

    // Iteration 0 is planned here; every later one was planned by the previous launch, during
    // its removal (the candidate order in f.sigma, the first wave in the control block).
    if (it == 0) {
        if (blockIdx.x == 0) plan_phase<Cfg::CONS, Cfg::TI, Cfg::TJ>(f, it, smem_raw, sh.red, f.sigma);
        if (!grid_sync(ctl, tmo)) return;
    }
    int chunk_base = 0;
    // phase times (opts.timing): CTA 0's global timer at the phase boundaries, which follow
    // grid barriers, so each interval covers the slowest CTA of the phase
    const bool timed = f.timing && blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long tph = timed ? global_ns() : 0;
    // the first wave as planned; later ones as published by each wave's finalisation
    Wave wv = {vc->ntiles, vc->ncol, vc->nrow};
    bool done = vc->done != 0;
    // wave words are numbered on from the last wave of the previous iteration
    for (unsigned seq = *reinterpret_cast<volatile unsigned*>(&ctl->seq0) + 1; !done; ++seq) {
        // opts.split_n caps the CTAs of the wave at split_n per tile (split_n = 1: each tile on
        // one CTA where the wave has fewer tiles than the grid has CTAs); 0 = the whole grid
        const long long gcap = f.split_n > 0 ? min((long long)gridDim.x, (long long)wv.ntiles * f.split_n)
                                             : (long long)gridDim.x;
        const Span sp = single_span((long long)wv.ntiles * (f.ld / kSub), gcap);
        // a narrow wave (16 columns or fewer) of the 64 x 32 kernel runs on 128 x 16 tiles,
        // compute and merge out of line
        bool narrow = false;
        if constexpr (std::is_same<Cfg, CfgF64>::value) narrow = wave_is_narrow(f.narrow, wv.ncol, wv.nrow);
        if (narrow) {
            if constexpr (std::is_same<Cfg, CfgF64>::value) {
                if (!narrow_wave<CfgN>(f, ctl, wv, sp, reinterpret_cast<float*>(ring), full, empty, sh, chunk_base,
                                       it, seq, tmo, timed, tph))
                    return;
            }
        } else {
            if (!compute_phase<Cfg>(f, ctl, wv, sp, ring, full, empty, sh, chunk_base)) {
                ctl->abort = 1;
                return;
            }
            if (!grid_sync(ctl, tmo)) return;
            if (timed) {
                const unsigned long long t = global_ns();
                ctl->phase_ns[0] += t - tph;
                tph = t;
            }
            merge_phase<Cfg>(f, wv, sp, it, sh, ring, seq);
        }
        fence_proxy_async();   // the merge used the copy ring as scratch
        // the wave's finalisation runs after every merge item, so its published word also
        // tells that every CTA is done with this wave's partial moments
        if (!wait_wave(ctl, seq, tmo, wv, done)) return;
        if (timed) {
            const unsigned long long t = global_ns();
            ctl->phase_ns[1] += t - tph;
            tph = t;
        }
    }
    if (it < f.p - 1) {
        iteration_tail<Cfg>(f, it, sh);
        if (timed) ctl->phase_ns[2] += global_ns() - tph;
    }
}

// ------------------------------------------------------------------ the batch kernel
// Many independent problems (datasets of uneven p and n, or bootstrap resamples) in one
// persistent cooperative launch: all iterations of all problems, in lockstep.  At
// iteration it every problem with p > it is planned by one CTA; each wave then
// concatenates the (tile, group) units of every problem whose iteration is not done
// and partitions them over the grid (stream-K across problems, so a wave of many
// small problems fills the GPU), merges each problem's tiles and runs its wave
// finalisation; the removals of all problems share the grid.  A problem whose status
// turns bad is not planned again (its outputs are not reported); a timeout or an
// abort ends the whole launch.
constexpr int kBatchMax = kBatchLaunchMax;   // problems per launch

struct BatchShared {
    long long uoff[kBatchMax + 1];   // first unit of each problem in this wave (prefix);
                                     // removal: first covariance element of each problem
    int ioff[kBatchMax + 1];         // first merge item of each problem in this wave;
                                     // removal: first row of each problem
    Wave wave[kBatchMax];            // each problem's wave, read at the wave's start
    int rr[kBatchMax];               // removal: rows of U (r) of each problem
    int root[kBatchMax];             // removal: each problem's root
    int fin[kBatchMax];              // merge: problems whose last item this CTA merged
    int nfin;
    unsigned char act[kBatchMax];    // per problem: take part in this phase (one read per CTA)
};

// Which problems a CTA-wide phase of iteration it covers, read once per CTA into shared
// memory so that every thread of the CTA takes the same branches (a problem's status can
// change while other CTAs work on it).  removal = 0: planned (p > it, status good);
// removal = 1: took a root this iteration and has rows left (it < p - 1).
__device__ void batch_active(const Fit* fits, int count, int it, int removal, BatchShared& bs) {
    for (int d = threadIdx.x; d < count; d += blockDim.x) {
        const Fit& f = fits[d];
        volatile Ctl* c = f.ctl;
        bool a = it < f.p && c->status == 0;
        if (removal) a = a && it < f.p - 1 && c->root >= 0;
        bs.act[d] = a ? 1 : 0;
    }
    __syncthreads();
}

// Block-wide exclusive prefix sum of one value per thread; the total to every thread.
template <int NTH>
__device__ __forceinline__ long long block_excl_scan(long long v, long long* lred, long long* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) lred[wid] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long run = 0;
        for (int w = 0; w < NTH / 32; ++w) {
            const long long t = lred[w];
            lred[w] = run;
            run += t;
        }
        lred[32] = run;
    }
    __syncthreads();
    const long long ex = lred[wid] + x - v;
    *total = lred[32];
    __syncthreads();
    return ex;
}

// The wave layout of all problems (every CTA computes the same one from the problems'
// control blocks, which change only in the merge phase, between two grid barriers).
template <int NTH, int TI>
__device__ void batch_layout(const Fit* fits, int count, int it, BatchShared& bs, IterShared& sh, long long& utot,
                             int& itot) {
    long long ubase = 0, ibase = 0;
    for (int base = 0; base < count; base += NTH) {
        const int d = base + int(threadIdx.x);
        long long u = 0, items = 0;
        if (d < count) {
            const Fit& f = fits[d];
            volatile Ctl* c = f.ctl;
            Wave w = {0, 0, 0};
            if (it < f.p && !c->done) {
                w = {c->ntiles, c->ncol, c->nrow};
                u = (long long)w.ntiles * (f.ld / kSub);
                items = (long long)w.ntiles * (NTH / 64);
            }
            bs.wave[d] = w;
        }
        long long tu, ti;
        const long long eu = block_excl_scan<NTH>(u, sh.lred, &tu);
        const long long ei = block_excl_scan<NTH>(items, sh.lred, &ti);
        if (d < count) {
            bs.uoff[d] = ubase + eu;
            bs.ioff[d] = int(ibase + ei);
        }
        ubase += tu;
        ibase += ti;
    }
    if (threadIdx.x == 0) {
        bs.uoff[count] = ubase;
        bs.ioff[count] = int(ibase);
    }
    __syncthreads();
    utot = ubase;
    itot = int(ibase);
}

// The last index d in [0, count) with off[d] <= v (off nondecreasing, off[0] = 0 <= v).
template <class I>
__device__ __forceinline__ int last_le(const I* off, int count, long long v) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((long long)off[mid] <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Batches on the FP32 path: the merge items of all problems, one warp per item.  A batch's
// tiles are shared by few CTAs each, so an item has few partial slots and a CTA-wide item
// would mostly wait on its round trips; here sixteen items per CTA proceed at once.  The
// arithmetic and its order are those of merge_item: the slots b_first + w, + NW, ... of
// each "virtual warp" w are summed in order, those sums in w order; lane L holds the
// values of the item's pairs 8 L ... 8 L + 7.  The warp that merges a problem's last item
// records the problem, and the CTA then runs those problems' wave finalisations.
template <class Cfg>
__device__ __noinline__ void batch_merge_warps(const Fit* fits, int count, BatchShared& bs, long long utot,
                                               long long G, int itot, int it, IterShared& sh, float* scratch) {
    constexpr int TI = Cfg::TI, TJ = Cfg::TJ, CONS = Cfg::CONS;
    constexpr int NW = CONS / 32, PARTS = CONS / 64;
    constexpr int HJ = TJ / 2, IR = 2 * (64 / HJ);   // rows of an item
    static_assert(std::is_same<typename Cfg::T, float>::value, "FP32 path");
    static_assert(IR <= 32 && TJ <= 32, "an item's rows and columns are lanes");
    static_assert(size_t(NW) * IR * (TJ + 1) * sizeof(float) <= ring_bytes<Cfg>(), "staging fits the ring");
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float* sI = scratch + wid * (IR * (TJ + 1));
    if (threadIdx.x == 0) bs.nfin = 0;
    __syncthreads();
    // Many items (at least half a warp each): consecutive items to the warps of a CTA (a
    // problem's items and finalisation stay together); fewer: item gi to warp gi / grid of
    // CTA gi mod grid, spread over all CTAs first.  The choice depends on itot alone.
    const bool blocked = itot >= int(gridDim.x) * NW / 2;
    for (int gi = blocked ? int(blockIdx.x) * NW + wid : wid * int(gridDim.x) + int(blockIdx.x); gi < itot;
         gi += gridDim.x * NW) {
        const int d = last_le(bs.ioff, count, gi);
        const Fit& f = fits[d];
        Ctl* ctl = f.ctl;
        const Wave wv = bs.wave[d];
        const int ncol = wv.ncol, nrow = wv.nrow;
        const long long off = bs.uoff[d];
        const int b_base = cta_of_unit(off, utot, G);
        const int item = gi - bs.ioff[d];
        const int t = item / PARTS, part = item % PARTS;
        const long long ng = f.ld / kSub;
        const int b_first = cta_of_unit(off + (long long)t * ng, utot, G) - b_base;
        const int b_last = cta_of_unit(off + (long long)(t + 1) * ng - 1, utot, G) - b_base;
        // this lane's pairs 8 lane + j: their rows, columns and variables
        int vi[8], vj[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int tp = 8 * lane + j;
            const int ct = part * 64 + (tp >> 2), q = tp & 3;
            const int e = t * TI + ct / HJ + (q >> 1) * (TI / 2), cc = ct % HJ + (q & 1) * HJ;
            vi[j] = e < nrow ? ld2(f.rows + e) : -1;
            vj[j] = cc < ncol ? ld2(f.cols + cc) : -1;
        }
        // 1. the item's 1024 values, 32 per lane, over its slots
        const float* parts = static_cast<const float*>(f.partials);
        const int b_stop = LINGAM_INBOUNDS(ctl, t + b_last < f.nslots) ? b_last : b_first - 1;
        float acc[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) acc[k] = 0.f;
        for (int w = 0; w < NW; ++w) {
            int bb = b_first + w;
            if (bb > b_stop) continue;   // an empty virtual warp adds +0: no change
            float vs[32];
            {
                const float* src = parts + ((size_t(t) + bb) * CONS + part * 64) * 16 + lane * 32;
                load16_cg(vs, src);
                load16_cg(vs + 16, src + 16);
            }
            for (bb += NW; bb <= b_stop; bb += NW) {
                const float* src = parts + ((size_t(t) + bb) * CONS + part * 64) * 16 + lane * 32;
                float v[32];
                load16_cg(v, src);
                load16_cg(v + 16, src + 16);
#pragma unroll
                for (int k = 0; k < 32; ++k) vs[k] += v[k];
            }
#pragma unroll
            for (int k = 0; k < 32; ++k) acc[k] += vs[k];
        }
        // 2. I of the lane's 8 pairs, staged by (item row, column)
        const float inv_n = __frcp_rn(float(f.n));
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int tp = 8 * lane + j;
            const int ct = part * 64 + (tp >> 2), q = tp & 3;
            const int e = t * TI + ct / HJ + (q >> 1) * (TI / 2), cc = ct % HJ + (q & 1) * HJ;
            bool okp = vi[j] >= 0 && vj[j] >= 0;
            if (okp) okp = f.reuse ? (e >= ncol || cc < e) : (vi[j] != vj[j]);
            float I = 0.f;
            if (okp) {
                I = pair_measure_f(acc[4 * j + 0], acc[4 * j + 1], acc[4 * j + 2], acc[4 * j + 3],
                                   __ldcg(f.vstat + vi[j]), __ldcg(f.vstat + vj[j]), inv_n);
                if (!isfinite(I)) set_status(ctl, LINGAM_EDEGENERATE);
            }
            const int el = ct / HJ - part * (64 / HJ) + (q >> 1) * (64 / HJ);
            sI[el * (TJ + 1) + cc] = I;
        }
        __syncwarp();
        // 3. the item's rows' contributions over all columns, and its part of each column's
        if (lane < IR) {
            const int e = t * TI + (lane < IR / 2 ? part * (IR / 2) + lane : part * (IR / 2) + lane - IR / 2 + TI / 2);
            FF a;
            for (int cc = 0; cc < TJ; ++cc) a.add_sq(fminf(sI[lane * (TJ + 1) + cc], 0.f));
            if (e < nrow) f.rowsum[e] = a.value();
        }
        if (lane < TJ) {
            FF a;
            for (int el = 0; el < IR; ++el) a.add_sq(fmaxf(sI[el * (TJ + 1) + lane], 0.f));
            reinterpret_cast<float2*>(f.colsum)[(size_t(t) * PARTS + part) * TJ + lane] = make_float2(a.hi, a.lo);
        }
        __threadfence();
        __syncwarp();
        if (lane == 0 && atomicAdd(&ctl->merged, 1) == wv.ntiles * PARTS - 1) bs.fin[atomicAdd(&bs.nfin, 1)] = d;
        __syncwarp();   // sI is staged again by the next item
    }
    __syncthreads();
    const int nfin = bs.nfin;
    for (int k = 0; k < nfin; ++k) {
        const int d = bs.fin[k];
        __threadfence();
        wave_finalize<CONS, TI, TJ>(fits[d], bs.wave[d], it, sh.red, 0u);
        __syncthreads();
    }
}

// The removal of every problem that took a root, spread over the whole grid at once (a
// CTA that walked the problems one after another would pay each problem's latency): the
// rows of U of all problems are numbered one after another, and so are the elements of
// their covariance blocks.  Every CTA computes the same numbering from the problems'
// control blocks, which the removal does not change.
template <int NTH>
__device__ void batch_removal_layout(const Fit* fits, int count, BatchShared& bs, IterShared& sh, int& rtot,
                                     long long& etot) {
    long long rbase = 0, ebase = 0;
    for (int base = 0; base < count; base += NTH) {
        const int d = base + int(threadIdx.x);
        long long rows = 0, elems = 0;
        if (d < count) {
            int r = 0, root = -1;
            if (bs.act[d]) {
                volatile Ctl* c = fits[d].ctl;
                r = c->r;
                root = c->root;
            }
            bs.rr[d] = r;
            bs.root[d] = root;
            rows = r;
            elems = (long long)r * r;
        }
        long long tr, te;
        const long long er = block_excl_scan<NTH>(rows, sh.lred, &tr);
        const long long ee = block_excl_scan<NTH>(elems, sh.lred, &te);
        if (d < count) {
            bs.ioff[d] = int(rbase + er);
            bs.uoff[d] = ebase + ee;
        }
        rbase += tr;
        ebase += te;
    }
    if (threadIdx.x == 0) {
        bs.ioff[count] = int(rbase);
        bs.uoff[count] = ebase;
    }
    __syncthreads();
    rtot = int(rbase);
    etot = ebase;
}

// UpdateData (Algorithm 7) with the new H(x_w), one warp per row of any problem.  On the
// FP32 path lanes take float4, sum the moments of 32 samples in FP32 and flush them into
// float-float sums, and the warp tree is float-float (FP64 adds are slow on this part).  The
// FP64 path sums single samples in FP64.
template <class Cfg>
__device__ __noinline__ void batch_remove_data(const Fit* fits, int count, const BatchShared& bs, int rtot) {
    using T = typename Cfg::T;
    constexpr int NW = Cfg::CONS / 32;
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * NW + (threadIdx.x >> 5), GW = gridDim.x * NW;
    for (int i = gw; i < rtot; i += GW) {
        const int d = last_le(bs.ioff, count, i);
        const Fit& f = fits[d];
        const int root = bs.root[d], p = f.p, ld = f.ld, n = f.n;
        const int w = ld2(f.sigma + (i - bs.ioff[d]));
        if (w == root) continue;
        const double c = f.sig[size_t(root) * p + w], inv = ld2(f.inv_root + w);
        T* xw = static_cast<T*>(f.xt) + size_t(w) * ld;
        const T* xr = static_cast<const T*>(f.xt) + size_t(root) * ld;
        double L = 0.0, Gs = 0.0;
        if constexpr (std::is_same<T, float>::value) {
            const float cc = float(c), ii = float(inv);
            float4* xw4 = reinterpret_cast<float4*>(xw);
            const float4* xr4 = reinterpret_cast<const float4*>(xr);
            const int n4 = ld / 4;
            float2 Lf = make_float2(0.f, 0.f), Gf = make_float2(0.f, 0.f);
            for (int b0 = lane; b0 < n4; b0 += 32 * 8) {
                float lcc = 0.f, g = 0.f;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int t4 = b0 + 32 * q;
                    if (t4 < n4) {
                        const float4 a = xw4[t4], rr = xr4[t4];
                        float4 o;
                        o.x = fmaf(-cc, rr.x, a.x) * ii;
                        o.y = fmaf(-cc, rr.y, a.y) * ii;
                        o.z = fmaf(-cc, rr.z, a.z) * ii;
                        o.w = fmaf(-cc, rr.w, a.w) * ii;
                        xw4[t4] = o;   // padding samples stay exactly zero
                        const int t = 4 * t4;
                        if (t + 0 < n) mom_add(o.x, lcc, g);
                        if (t + 1 < n) mom_add(o.y, lcc, g);
                        if (t + 2 < n) mom_add(o.z, lcc, g);
                        if (t + 3 < n) mom_add(o.w, lcc, g);
                    }
                }
                Lf = ff_add(Lf, make_float2(lcc, 0.f));
                Gf = ff_add(Gf, make_float2(g, 0.f));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                Lf = ff_add(Lf, make_float2(__shfl_xor_sync(0xffffffffu, Lf.x, o), __shfl_xor_sync(0xffffffffu, Lf.y, o)));
                Gf = ff_add(Gf, make_float2(__shfl_xor_sync(0xffffffffu, Gf.x, o), __shfl_xor_sync(0xffffffffu, Gf.y, o)));
            }
            L = double(Lf.x) + double(Lf.y);
            Gs = double(Gf.x) + double(Gf.y);
        } else {
            for (int t = lane; t < ld; t += 32) {
                const double u = fma(-c, xr[t], xw[t]) * inv;
                xw[t] = u;
                if (t < n) mom_add(u, L, Gs);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                L += __shfl_xor_sync(0xffffffffu, L, o);
                Gs += __shfl_xor_sync(0xffffffffu, Gs, o);
            }
        }
        if (lane == 0) {
            f.hx[w] = hterm_inv(L, Gs, f.inv_n);
            f.vstat[w] = var_stats_inv(L, Gs, n, ld, f.inv_n);
        }
    }
}

// UpdateCovMat (Algorithm 8 / Eq. CovUpdate) in FP64, one thread per element (w, j) of
// any problem's block of U without its root.
template <class Cfg>
__device__ __noinline__ void batch_remove_cov(const Fit* fits, int count, const BatchShared& bs, long long etot) {
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x, GT = (long long)gridDim.x * blockDim.x;
    for (long long e = gt; e < etot; e += GT) {
        const int d = last_le(bs.uoff, count, e);
        const Fit& f = fits[d];
        const int r = bs.rr[d], root = bs.root[d], p = f.p;
        const long long loc = e - bs.uoff[d];
        const int kk = int(loc / r), jj = int(loc - (long long)kk * r);
        const int w = ld2(f.sigma + kk), j = ld2(f.sigma + jj);
        if (w == root || j == root) continue;
        double* row = f.sig + size_t(w) * p;
        double nv = 1.0;
        if (j != w) {
            const double* rootrow = f.sig + size_t(root) * p;
            nv = (row[j] - rootrow[w] * rootrow[j]) * (ld2(f.inv_root + w) * ld2(f.inv_root + j));
        }
        row[j] = nv;
        if (f.precision == LINGAM_MIXED) f.sigf[size_t(w) * p + j] = sig_pair_f(nv);
    }
}

template <class Cfg>
__global__ void __launch_bounds__(Cfg::CONS, Cfg::MINB) k_batch(const Fit* __restrict__ fits, int count, int maxp,
                                                               Ctl* bctl) {
    unsigned char* smem_raw = smem_dyn;
    __shared__ IterShared sh;
    __shared__ BatchShared bs;
    using T = typename Cfg::T;
    constexpr int CONS = Cfg::CONS, TI = Cfg::TI;
    T* ring = reinterpret_cast<T*>(smem_raw);
    const size_t ring_or_sort =
        ring_bytes<Cfg>() > size_t(sort_max<Cfg>()) * 8 ? ring_bytes<Cfg>() : size_t(sort_max<Cfg>()) * 8;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + ring_or_sort);
    uint64_t* empty = full + kStages;
    volatile Ctl* vb = bctl;
    if (vb->status != 0) return;
    const unsigned long long tmo = vb->timeout_ns;
    if (threadIdx.x == 0) {
        for (int s = 0; s < Cfg::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], Cfg::CONS / 32);
        }
        sh.abort = 0;
        fence_barrier_init();
    }
    __syncthreads();
    int chunk_base = 0;   // ring position, continued over all waves of the launch
    for (int it = 0; it < maxp; ++it) {
        // plan (a problem whose status turned bad stays done: it is not planned again)
        batch_active(fits, count, it, 0, bs);
        for (int d = blockIdx.x; d < count; d += gridDim.x)
            if (bs.act[d]) plan_phase<CONS, TI, Cfg::TJ, sort_max<Cfg>()>(fits[d], it, smem_raw, sh.red, fits[d].sigma);
        if (!grid_sync(bctl, tmo)) return;
        for (;;) {
            long long utot;
            int itot;
            batch_layout<CONS, TI>(fits, count, it, bs, sh, utot, itot);
            if (utot == 0) break;
            const long long G = working_ctas(utot, gridDim.x);
            const int b = blockIdx.x;
            if (b < G) {
                const long long lo = unit_lo(b, utot, G), hi = unit_lo(b + 1, utot, G);
                for (int d = last_le(bs.uoff, count, lo); d < count && bs.uoff[d] < hi; ++d) {
                    if (bs.uoff[d + 1] == bs.uoff[d]) continue;   // no units this wave
                    const Span sp{bs.uoff[d], utot, G, cta_of_unit(bs.uoff[d], utot, G)};
                    if (!compute_phase<Cfg>(fits[d], bctl, bs.wave[d], sp, ring, full, empty, sh, chunk_base)) {
                        bctl->abort = 1;
                        return;
                    }
                }
            }
            if (!grid_sync(bctl, tmo)) return;
            if constexpr (std::is_same<T, float>::value) {
                batch_merge_warps<Cfg>(fits, count, bs, utot, G, itot, it, sh, ring);
            } else {
                for (int gi = blockIdx.x; gi < itot; gi += gridDim.x) {
                    const int d = last_le(bs.ioff, count, gi);
                    const Span sp{bs.uoff[d], utot, G, cta_of_unit(bs.uoff[d], utot, G)};
                    merge_item<Cfg>(fits[d], bs.wave[d], sp, it, sh, ring, gi - bs.ioff[d], 0u);
                }
            }
            fence_proxy_async();   // the merge used the copy ring as scratch
            if (!grid_sync(bctl, tmo)) return;
        }
        // UpdateData and UpdateCovMat of every problem that took a root, all problems' rows
        // and covariance elements spread over the grid at once (disjoint memory: the root's
        // row and column, from which the coefficients come, are not written)
        batch_active(fits, count, it, 1, bs);
        int rtot;
        long long etot;
        batch_removal_layout<CONS>(fits, count, bs, sh, rtot, etot);
        batch_remove_data<Cfg>(fits, count, bs, rtot);
        batch_remove_cov<Cfg>(fits, count, bs, etot);
        if (!grid_sync(bctl, tmo)) return;
    }
}

// ------------------------------------------------------------------ batches: one pair per warp
// The pair mode of the batch kernel, for many small problems: a wave's needed pairs (its
// columns against each other and against the other rows, Sec. III-A) are enumerated and each
// is evaluated whole by one warp, so no pair slot of a tile is computed in vain.
// The per-sample arithmetic, the group closing and the pair measure are the tile path's; the
// lanes' group sums are added in a tree.  Each problem's pair measures go to its I buffer; one CTA per
// problem then sums its rows' and columns' contributions in a fixed order and runs the wave
// finalisation.  Waves have up to kPairTJ columns; a wave has one nominal "tile" of kPairTI
// rows (the finalisation's column parts: part 0 holds the sums, the others stay zero).
constexpr int kPairTJ = 16;
constexpr int kPairTI = 1024;
constexpr int kPairThr = 256;

// Unordered pair q of a wave with ncol columns and nrow rows (columns first): column c of
// row slot e, for c < ncol <= e (the columns against the other rows), then c < e < ncol
// (the columns' own triangle).
__device__ __forceinline__ void pair_of(long long q, int ncol, int nrow, int& e, int& c) {
    const int qq = int(q);   // below ncol * nrow <= kPairTJ * 16384
    const int cross = ncol * (nrow - ncol);
    if (qq < cross) {
        const int k = qq / ncol;
        e = ncol + k;
        c = qq - k * ncol;
    } else {
        const int t = qq - cross;   // triangle index: e (e - 1) / 2 + c, c < e < ncol <= kPairTJ
        int ee = 1;
        while ((ee + 1) * ee / 2 <= t) ++ee;
        e = ee;
        c = t - ee * (ee - 1) / 2;
    }
}
__device__ __forceinline__ long long wave_pairs(int ncol, int nrow) {
    return (long long)ncol * (ncol - 1) / 2 + (long long)ncol * (nrow - ncol);
}

// Closes one 32-sample group of both directions into the lane's sums (the tile path's group
// closing: one lg2 of the product, the centring offset .w of each variable).
__device__ __forceinline__ void close_group(const Acc2& aa, const Acc2& ab, float4 si, float4 sj, float& Da,
                                            float& Ga, float& Db, float& Gb) {
    Da += fmaf(float(kLn2), lg2_approx(aa.P.x * aa.P.y), fmaf(aa.A.x + aa.A.y, kInvScale / -kC3, si.w));
    Ga += aa.G.x + aa.G.y;
    Db += fmaf(float(kLn2), lg2_approx(ab.P.x * ab.P.y), fmaf(ab.A.x + ab.A.y, kInvScale / -kC3, sj.w));
    Gb += ab.G.x + ab.G.y;
}
__device__ __forceinline__ void acc_pair4(Acc2& aa, Acc2& ab, float4 a4, float4 b4, float2 s2, float2 sr2) {
    const float2 vi2[2] = {make_float2(a4.x, a4.y), make_float2(a4.z, a4.w)};
    const float2 vj2[2] = {make_float2(b4.x, b4.y), make_float2(b4.z, b4.w)};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        acc2_add(aa, __ffma2_rn(s2, vi2[h], __fmul2_rn(sr2, vj2[h])));
        acc2_add(ab, __ffma2_rn(s2, vj2[h], __fmul2_rn(sr2, vi2[h])));
    }
}
__device__ __forceinline__ void acc_init(Acc2& a) {
    a.A = make_float2(0.f, 0.f);
    a.P = make_float2(1.f, 1.f);
    a.G = make_float2(0.f, 0.f);
}

// One pair (row variable vi, column variable vj) by a whole warp; the measure I to every lane.
// A 32-sample group of a lane is any 32 of the row's samples (the centring offset is per group
// and the padding samples are zero), so the reads are coalesced: in each block of 1024
// samples lane l takes the four samples 4l .. 4l + 3 of each 128-sample chunk, eight chunks
// making its group.  The rows' last ld mod 1024 samples (a multiple of 128) are closed as
// whole 32-sample groups, one per lane.
__device__ __forceinline__ float pair_by_warp(const Fit& f, int vi, int vj, bool& degenerate) {
    const int lane = threadIdx.x & 31;
    const int p = f.p, ld = f.ld;
    float2 ro = __ldcg(f.sigf + size_t(vi) * p + vj);
    degenerate = !(ro.y > float(degenerate_om(true)));
    if (degenerate) ro = make_float2(0.f, 1.f);
    const float sc = kScale / sqrtf(ro.y);
    const float2 s2 = make_float2(sc, sc), sr2 = make_float2(-sc * ro.x, -sc * ro.x);
    const float4 si = __ldcg(f.vstat + vi), sj = __ldcg(f.vstat + vj);
    const float* xi = static_cast<const float*>(f.xt) + size_t(vi) * ld;
    const float* xj = static_cast<const float*>(f.xt) + size_t(vj) * ld;
    float Da = 0.f, Ga = 0.f, Db = 0.f, Gb = 0.f;
    const int nblk = ld >> 10;
    for (int b = 0; b < nblk; ++b) {
        const float4* ri = reinterpret_cast<const float4*>(xi + (size_t(b) << 10)) + lane;
        const float4* rj = reinterpret_cast<const float4*>(xj + (size_t(b) << 10)) + lane;
        float4 a4[8], b4[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            a4[k] = ri[32 * k];
            b4[k] = rj[32 * k];
        }
        Acc2 aa, ab;
        acc_init(aa);
        acc_init(ab);
#pragma unroll
        for (int k = 0; k < 8; ++k) acc_pair4(aa, ab, a4[k], b4[k], s2, sr2);
        close_group(aa, ab, si, sj, Da, Ga, Db, Gb);
    }
    const int g = (nblk << 5) + lane;   // tail: one contiguous group per lane
    if (g < ld / kSub) {
        const float4* ri = reinterpret_cast<const float4*>(xi + size_t(g) * kSub);
        const float4* rj = reinterpret_cast<const float4*>(xj + size_t(g) * kSub);
        Acc2 aa, ab;
        acc_init(aa);
        acc_init(ab);
#pragma unroll 4
        for (int k = 0; k < kSub / 4; ++k) acc_pair4(aa, ab, ri[k], rj[k], s2, sr2);
        close_group(aa, ab, si, sj, Da, Ga, Db, Gb);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Da += __shfl_xor_sync(0xffffffffu, Da, o);
        Ga += __shfl_xor_sync(0xffffffffu, Ga, o);
        Db += __shfl_xor_sync(0xffffffffu, Db, o);
        Gb += __shfl_xor_sync(0xffffffffu, Gb, o);
    }
    return pair_measure_f(Da, Ga, Db, Gb, si, sj, __frcp_rn(float(f.n)));
}

// One problem's wave after its pairs: the rows' contributions sum_c min(0, I)^2 (a thread per
// row) and the columns' sum_e max(0, I)^2 (a warp per column, lanes over the rows, then a
// tree), float-float in a fixed order, into the buffers the finalisation reads.
template <int NTH>
__device__ void pairs_merge(const Fit& f, const Wave& wv) {
    const int ncol = wv.ncol, nrow = wv.nrow, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const float* I = static_cast<const float*>(f.ibuf);
    for (int e = tid; e < nrow; e += NTH) {
        FF acc;
        const int cmax = e < ncol ? e : ncol;   // the pairs of row slot e
        for (int c = 0; c < cmax; ++c) acc.add_sq(fminf(I[size_t(e) * kPairTJ + c], 0.f));
        f.rowsum[e] = acc.value();
    }
    constexpr int PARTS = NTH / 64;
    const int nparts = wv.ntiles * PARTS;
    for (int c = wid; c < kPairTJ; c += NTH / 32) {
        FF acc;
        if (c < ncol)
            for (int e = c + 1 + lane; e < nrow; e += 32) acc.add_sq(fmaxf(I[size_t(e) * kPairTJ + c], 0.f));
        float2 v = make_float2(acc.hi, acc.lo);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float2 w = make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
            v = ff_add(v, w);
        }
        for (int at = lane; at < nparts; at += 32) {
            const float2 ff = at == 0 ? v : make_float2(0.f, 0.f);
            f.colsum[size_t(at) * kPairTJ + c] = *reinterpret_cast<const double*>(&ff);
        }
    }
}

// Every needed pair of every problem's wave, one warp per pair, into the problems' I
// buffers.  Out of line, so that the sample loop's registers are allocated apart from the
// rest of the kernel.
__device__ __noinline__ void pairs_compute(const Fit* __restrict__ fits, int count, const BatchShared& bs,
                                           long long ptot) {
    constexpr int NW = kPairThr / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (long long g = (long long)blockIdx.x * NW + wid; g < ptot; g += (long long)gridDim.x * NW) {
        const int d = last_le(bs.uoff, count, g);
        const Fit& f = fits[d];
        const Wave wv = bs.wave[d];
        int e, c;
        pair_of(g - bs.uoff[d], wv.ncol, wv.nrow, e, c);
        bool degenerate;
        const float I = pair_by_warp(f, ld2(f.rows + e), ld2(f.cols + c), degenerate);
        if (lane == 0) {
            if (degenerate || !isfinite(I)) set_status(f.ctl, LINGAM_EDEGENERATE);
            static_cast<float*>(f.ibuf)[size_t(e) * kPairTJ + c] = I;
        }
    }
}

__global__ void __launch_bounds__(kPairThr, 2) k_batch_pairs(const Fit* __restrict__ fits, int count, int maxp,
                                                             Ctl* bctl) {
    unsigned char* smem_raw = smem_dyn;
    __shared__ IterShared sh;
    __shared__ BatchShared bs;
    volatile Ctl* vb = bctl;
    if (vb->status != 0) return;
    const unsigned long long tmo = vb->timeout_ns;
    for (int it = 0; it < maxp; ++it) {
        batch_active(fits, count, it, 0, bs);
        for (int d = blockIdx.x; d < count; d += gridDim.x)
            if (bs.act[d]) plan_phase<kPairThr, kPairTI, kPairTJ, 2048>(fits[d], it, smem_raw, sh.red, fits[d].sigma);
        if (!grid_sync(bctl, tmo)) return;
        for (;;) {
            // the wave of every problem whose iteration is not done, and its pairs' offsets
            // (a wave may have no pair left to evaluate, one column whose partners were all
            // columns before: it is still finalised)
            long long pbase = 0, nact = 0;
            for (int base = 0; base < count; base += kPairThr) {
                const int d = base + int(threadIdx.x);
                long long q = 0, a = 0;
                if (d < count) {
                    const Fit& f = fits[d];
                    volatile Ctl* c = f.ctl;
                    Wave w = {0, 0, 0};
                    if (it < f.p && !c->done && c->status == 0) {
                        w = {c->ntiles, c->ncol, c->nrow};
                        q = wave_pairs(w.ncol, w.nrow);
                        a = 1;
                    }
                    bs.wave[d] = w;
                    bs.act[d] = (unsigned char)a;
                }
                long long tq, ta;
                const long long eq = block_excl_scan<kPairThr>(q, sh.lred, &tq);
                block_excl_scan<kPairThr>(a, sh.lred, &ta);
                if (d < count) bs.uoff[d] = pbase + eq;
                pbase += tq;
                nact += ta;
            }
            if (threadIdx.x == 0) bs.uoff[count] = pbase;
            __syncthreads();
            const long long ptot = bs.uoff[count];
            if (nact == 0) break;
            pairs_compute(fits, count, bs, ptot);   // every needed pair of every problem
            if (!grid_sync(bctl, tmo)) return;
            // each problem's sums and finalisation, one CTA per problem
            for (int d = blockIdx.x; d < count; d += gridDim.x) {
                if (!bs.act[d]) continue;
                pairs_merge<kPairThr>(fits[d], bs.wave[d]);
                __syncthreads();   // the sums precede the finalisation's reads (same CTA)
                wave_finalize<kPairThr, kPairTI, kPairTJ>(fits[d], bs.wave[d], it, sh.red, 0u);
                __syncthreads();
            }
            if (!grid_sync(bctl, tmo)) return;
        }
        // UpdateData and UpdateCovMat of every problem that took a root (the tile path's)
        batch_active(fits, count, it, 1, bs);
        int rtot;
        long long etot;
        batch_removal_layout<kPairThr>(fits, count, bs, sh, rtot, etot);
        batch_remove_data<CfgF16>(fits, count, bs, rtot);
        batch_remove_cov<CfgF16>(fits, count, bs, etot);
        if (!grid_sync(bctl, tmo)) return;
    }
}

static cudaError_t launch_batch_pairs(const Fit* fits_dev, int count, int maxp, Ctl* bctl, int nsm, cudaStream_t st) {
    const size_t smem = size_t(2048) * sizeof(unsigned long long);   // the candidate sort
    cudaError_t e = ensure_smem_attr(reinterpret_cast<const void*>(k_batch_pairs), smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_pairs, kPairThr, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    cudaLaunchConfig_t cfg = {};
    const int grid = nsm * (per_sm < 2 ? per_sm : 2);
    cfg.gridDim = dim3(grid < kMaxGrid ? grid : kMaxGrid);
    cfg.blockDim = dim3(kPairThr);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batch_pairs, fits_dev, count, maxp, bctl);
}

// ------------------------------------------------------------------ host side
template <class Cfg>
static int grid_for(int nsm) {
    int per_sm = 0;
    const size_t smem = iter_smem_bytes<Cfg>();
    if (ensure_smem_attr(reinterpret_cast<const void*>(k_iteration<Cfg>), smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_iteration<Cfg>, Cfg::CONS, smem) != cudaSuccess)
        return 0;
    if (per_sm < 1) return 0;
    const int grid = nsm * (per_sm < Cfg::MINB ? per_sm : Cfg::MINB);   // all CTAs co-resident
    return grid < kMaxGrid ? grid : kMaxGrid;   // the workspace holds partial slots for kMaxGrid CTAs
}

int iteration_grid(const Fit& f, int nsm) {
    if (f.precision != LINGAM_MIXED) return grid_for<CfgD>(nsm);
    if (f.tile_cols == 16) return grid_for<CfgF16>(nsm);
    return f.tile_rows == 32 ? grid_for<CfgF32>(nsm) : grid_for<CfgF64>(nsm);
}

template <class Cfg>
static cudaError_t launch_iter(const Fit& f, int it, int grid, cudaStream_t st) {
    const size_t smem = iter_smem_bytes<Cfg>();
    cudaError_t e = ensure_smem_attr(reinterpret_cast<const void*>(k_iteration<Cfg>), smem);
    if (e != cudaSuccess) return e;
    Fit fc = f;
    void* args[] = {&fc, &it};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_iteration<Cfg>), dim3(grid), dim3(Cfg::CONS),
                                       args, smem, st);
}

cudaError_t launch_iteration(const Fit& f, int it, int grid, cudaStream_t st) {
    if (f.precision != LINGAM_MIXED) return launch_iter<CfgD>(f, it, grid, st);
    if (f.tile_cols == 16) return launch_iter<CfgF16>(f, it, grid, st);
    return f.tile_rows == 32 ? launch_iter<CfgF32>(f, it, grid, st) : launch_iter<CfgF64>(f, it, grid, st);
}

template <class Cfg>
static cudaError_t launch_batch_cfg(const Fit* fits_dev, int count, int maxp, Ctl* bctl, int nsm, cudaStream_t st) {
    const size_t smem = iter_smem_bytes<Cfg>();
    cudaError_t e = ensure_smem_attr(reinterpret_cast<const void*>(k_batch<Cfg>), smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<Cfg>, Cfg::CONS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    cudaLaunchConfig_t cfg = {};
    const int grid = nsm * (per_sm < Cfg::MINB ? per_sm : Cfg::MINB);
    cfg.gridDim = dim3(grid < kMaxGrid ? grid : kMaxGrid);   // partial slots exist for kMaxGrid CTAs
    cfg.blockDim = dim3(Cfg::CONS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batch<Cfg>, fits_dev, count, maxp, bctl);
}

cudaError_t launch_batch(const Fit* fits_dev, int count, int maxp, int precision, int tile_rows, int tile_cols,
                         Ctl* bctl, int nsm, cudaStream_t st) {
    if (count < 1 || count > kBatchMax) return cudaErrorInvalidValue;
    if (precision != LINGAM_MIXED) return launch_batch_cfg<CfgD>(fits_dev, count, maxp, bctl, nsm, st);
    if (tile_rows == 64 && tile_cols == 32) return launch_batch_cfg<CfgF64>(fits_dev, count, maxp, bctl, nsm, st);
    if (tile_rows == 64 && tile_cols == 16) return launch_batch_cfg<CfgF16>(fits_dev, count, maxp, bctl, nsm, st);
    if (tile_rows == 32 && tile_cols == 32) return launch_batch_cfg<CfgF32>(fits_dev, count, maxp, bctl, nsm, st);
    if (tile_rows == 32 && tile_cols == 16) return launch_batch_cfg<CfgB>(fits_dev, count, maxp, bctl, nsm, st);
    if (tile_rows == 1 && tile_cols == 1) return launch_batch_pairs(fits_dev, count, maxp, bctl, nsm, st);
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ bounded-wait self-test
// Each kind of device-side wait of the library, made to wait for something that never
// happens, must give up after the control block's timeout with LINGAM_ETIMEOUT recorded and
// let the kernel end normally: which = 0, an mbarrier phase that no thread completes (the
// copy-ring waits of the iteration and batch kernels); 1, a grid barrier whose arrival count
// starts one off, so that the second of two CTAs waits for an arrival that never comes (the
// iteration and batch kernels' barriers); 2, a wave word that nothing publishes; 3, a B-fit
// row flag that nothing sets (the Cholesky's data flow).
// No copies or tensor-memory allocations are in flight in this kernel.
__device__ Ctl g_selftest_ctl;
__device__ int g_selftest_flag;   // stays 0: the readiness flag nothing sets

__global__ void k_wait_selftest(int which) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_abort;
    Ctl* ctl = &g_selftest_ctl;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        s_abort = 0;
        fence_barrier_init();
    }
    __syncthreads();
    const unsigned long long tmo = *reinterpret_cast<volatile unsigned long long*>(&ctl->timeout_ns);
    if (which == 0) {
        mbar_wait_or_abort(&bar, 0, ctl, tmo, &s_abort);
    } else if (which == 1) {
        grid_sync(ctl, tmo);
    } else if (which == 3) {
        if (threadIdx.x == 0) wait_flag_set(&g_selftest_flag, ctl);
    } else {
        Wave wv;
        bool done = false;
        wait_wave(ctl, 1u, tmo, wv, done);
    }
}

cudaError_t run_wait_selftest(int which, unsigned long long timeout_ns, int* status, cudaStream_t st) {
    Ctl h = {};
    h.timeout_ns = timeout_ns;
    if (which == 1) h.bar_count = 1;   // one arrival off: the second CTA's block never fills
    const int zero = 0;
    cudaError_t ez = cudaMemcpyToSymbolAsync(g_selftest_flag, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, st);
    if (ez != cudaSuccess) return ez;
    cudaError_t e = cudaMemcpyToSymbolAsync(g_selftest_ctl, &h, sizeof(h), 0, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    k_wait_selftest<<<which == 1 ? 2 : 1, 32, 0, st>>>(which);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemcpyFromSymbolAsync(&h, g_selftest_ctl, sizeof(h), 0, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    *status = h.status;
    return cudaSuccess;
}

}  // namespace lingam

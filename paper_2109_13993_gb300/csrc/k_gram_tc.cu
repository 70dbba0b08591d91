// k_gram_tc.cu -- CalculateCovMat (Algorithm 3) of the mixed path on the
// tensor cores: Sigma = Xn Xn^T / (n-1) for the normalised FP32 rows Xn.
//
// Error-free splitting (the scheme of Ozaki, Ogita, Oishi and Rump, 2012):
// each row i is scaled by a power of two 2^-e_i so that |y| < 1, and
// y 2^7 = D0 + 2^-7 D1 + 2^-14 T with D0, D1 integers (|D0| <= 128,
// |D1| <= 64) and T the TF32 rounding of the remaining tail (|T| <= 64); all
// three are exact TF32 operands.  Then
//   x_i x_j 2^(14 - e_i - e_j) = D0D0 + 2^-7 (D0D1 + D1D0)
//                              + 2^-14 (D0T + TD0 + D1D1) + 2^-21 (D1T + TD1) + O(2^-28 TT),
// and the four levels accumulate in four tensor-memory accumulators (the
// whole 512-column TMEM).  The products of the first two levels are integers
// of at most 2^14, so their FP32 sums stay exact for 512 samples whatever the
// rounding of the tensor core's adder; the last two levels carry weights of
// 2^-14 and 2^-21, so their FP32 rounding is negligible.  Every 512 samples
// the accumulators are drained into float-float sums in registers.  The
// split of the sample axis over CTAs is summed in FP64 by a second kernel,
// which also applies 2^(e_i + e_j - 14) / (n - 1).
//
// Per CTA (320 threads): warp 8 streams the six 128 x 32 operand blocks of a
// k-step (D0, D1, T of the row tile and of the column tile) into a two-stage
// shared-memory ring with 2-D TMA loads (128-byte swizzle); warp 9 issues the
// tcgen05.mma instructions (kind::tf32, M = N = 128, K = 8) that read the ring
// through shared-memory matrix descriptors, and commits each stage back to
// the producer; warps 0-7 drain the accumulators (warp w reads TMEM lanes
// 32 (w mod 4) ... and columns 64 (w / 4) ... of each level).  All waits are
// bounded by the fit's timeout.
#include <cuda.h>

#include "common.cuh"
#include "launch.h"
#include "tma.cuh"

namespace lingam {

constexpr int kGM = 128;                          // tile rows = tile columns
constexpr int kGKB = 32;                          // samples per k-step (128 bytes of FP32)
constexpr int kGStagesTC = 2;
constexpr int kGOps = 6;                          // operand blocks per stage
constexpr uint32_t kGBlockBytes = kGM * kGKB * 4;  // one 128 x 32 operand block, 16 KB
constexpr uint32_t kGStageBytes = kGOps * kGBlockBytes;
constexpr int kGDrain = 16;                       // k-steps (512 samples) per accumulation group
constexpr int kGDrainWarps = 8;
constexpr int kGThreads = 32 * (kGDrainWarps + 2);
constexpr uint32_t kGTmemCols = 4 * kGM;          // four level accumulators

__host__ __device__ constexpr size_t gram_tc_smem_bytes() { return size_t(kGStagesTC) * kGStageBytes + 1024; }

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {   // whole warp
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {   // whole warp
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {   // whole warp
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[desc] * B[desc]^T, both K-major, TF32 inputs, FP32 accumulator.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// Arrive on `bar` once every tcgen05.mma issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// 8 consecutive accumulator columns of two accumulators (TMEM addresses ta, tb) of this
// warp's 32 lanes (one row per thread), both loads in flight before one wait.
__device__ __forceinline__ void tmem_ld8x2(uint32_t ta, uint32_t tb, float* va, float* vb) {
    uint32_t a[8], b[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7])
                 : "r"(ta));
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3]), "=r"(b[4]), "=r"(b[5]), "=r"(b[6]), "=r"(b[7])
                 : "r"(tb));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        va[k] = __uint_as_float(a[k]);
        vb[k] = __uint_as_float(b[k]);
    }
}
// 2-D TMA load of one box (x = innermost coordinate in elements) into shared memory.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major operand block stored with the
// 128-byte swizzle (rows of 128 bytes, 8-row atoms 1024 bytes apart).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t smem_addr) {
    uint64_t d = 0;
    d |= uint64_t((smem_addr & 0x3FFFFu) >> 4);   // start address
    d |= uint64_t(16 >> 4) << 16;                 // leading-dimension byte offset (unused with this swizzle)
    d |= uint64_t(1024 >> 4) << 32;               // stride-dimension byte offset: 8 rows x 128 bytes
    d |= uint64_t(1) << 46;                       // descriptor version for tcgen05
    d |= uint64_t(2) << 61;                       // 128-byte swizzle
    return d;
}
// Instruction descriptor: D FP32, A and B TF32, both K-major, M = N = 128.
constexpr uint32_t kIdescTF32 = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(kGM >> 3) << 17) |
                                (uint32_t(kGM >> 4) << 24);

__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, Ctl* ctl, unsigned long long tmo) {
    return mbar_wait_bounded(bar, parity, ctl, tmo);
}

// Knuth's TwoSum: s + e == a + b exactly (round-to-nearest, no contraction).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// ------------------------------------------------------------------ digits of the normalised rows
// One CTA per row: e = the exponent of max_t |x_t| (so |x 2^-e| < 1), then the
// digits D0, D1 and the TF32 tail T of y 2^7 = x 2^(7-e), written as FP32.
constexpr int kDigitThreads = 256;
__global__ void __launch_bounds__(kDigitThreads) k_digits(const float* __restrict__ x, float* __restrict__ d0,
                                                        float* __restrict__ d1, float* __restrict__ tt,
                                                        int* __restrict__ expo, int ld) {
    __shared__ float red[kDigitThreads / 32];
    const size_t row = size_t(blockIdx.x) * ld;
    float m = 0.f;
    for (int t = threadIdx.x * 4; t < ld; t += kDigitThreads * 4) {
        const float4 v = *reinterpret_cast<const float4*>(x + row + t);
        m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    m = red[0];
#pragma unroll
    for (int w = 1; w < kDigitThreads / 32; ++w) m = fmaxf(m, red[w]);
    int e = 0;
    frexpf(m, &e);   // m = f 2^e, f in [0.5, 1) (e = 0 for m = 0)
    if (threadIdx.x == 0) expo[blockIdx.x] = e;
    for (int t = threadIdx.x; t < ld; t += kDigitThreads) {
        const float y = ldexpf(x[row + t], 7 - e);   // exact: a power-of-two scaling
        const float a = rintf(y);
        const float r0 = ldexpf(y - a, 7);            // y - a is exact, |y - a| <= 1/2
        const float b = rintf(r0);
        const float r1 = ldexpf(r0 - b, 7);
        const float c = __uint_as_float((__float_as_uint(r1) + 0x1000u) & 0xFFFFE000u);   // TF32 rounding
        d0[row + t] = a;
        d1[row + t] = b;
        tt[row + t] = c;
    }
}

// ------------------------------------------------------------------ the tensor-core Gram
struct GramMaps {
    CUtensorMap d0, d1, tt;
};

__global__ void __launch_bounds__(kGThreads, 1)
    k_gram_tc(const __grid_constant__ GramMaps maps, float2* __restrict__ partial, int nt, int kb_per_split,
              int kb_total, int nsplit, Ctl* ctl) {
    extern __shared__ unsigned char smem_dyn[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full[kGStagesTC], empty[kGStagesTC], tfull, tempty;
    __shared__ uint32_t tmem_base;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = blockIdx.x / nsplit, split = blockIdx.x % nsplit;
    int bi = 0, rem = tile;
    while (rem >= nt - bi) {
        rem -= nt - bi;
        ++bi;
    }
    const int bj = bi + rem;
    const int kb0 = split * kb_per_split;
    const int nkb = max(0, min(kb_total, kb0 + kb_per_split) - kb0);
    const int ngroups = (nkb + kGDrain - 1) / kGDrain;
    const unsigned long long tmo = ctl->timeout_ns;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kGStagesTC; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&tfull, 1);
        mbar_init(&tempty, kGDrainWarps);   // one arrival per draining warp
        fence_barrier_init();
    }
    if (warp == 0) {
        tmem_alloc(&tmem_base, kGTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == kGDrainWarps) {
        if (lane == 0) {   // producer: D0, D1, T of the row tile bi, then of the column tile bj
            const CUtensorMap* mp[3] = {&maps.d0, &maps.d1, &maps.tt};
            for (int k = 0; k < nkb; ++k) {
                const int s = k % kGStagesTC;
                if (k >= kGStagesTC && !wait_bar(&empty[s], ((k / kGStagesTC) - 1) & 1, ctl, tmo)) break;
                unsigned char* st = smem + size_t(s) * kGStageBytes;
                mbar_expect_tx(&full[s], kGStageBytes);
                const int x = (kb0 + k) * kGKB;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    tma_load_2d(st + q * kGBlockBytes, mp[q], x, bi * kGM, &full[s]);
                    tma_load_2d(st + (3 + q) * kGBlockBytes, mp[q], x, bj * kGM, &full[s]);
                }
            }
        }
        __syncwarp();
    } else if (warp == kGDrainWarps + 1) {
        if (lane == 0) {   // MMA issuer
            for (int k = 0; k < nkb; ++k) {
                const int s = k % kGStagesTC;
                const int g = k / kGDrain;
                const bool first = (k % kGDrain) == 0;
                if (first && g >= 1 && !wait_bar(&tempty, (g - 1) & 1, ctl, tmo)) break;
                if (!wait_bar(&full[s], (k / kGStagesTC) & 1, ctl, tmo)) break;
                tc_fence_after();
                const uint32_t base = smem_u32(smem + size_t(s) * kGStageBytes);
#pragma unroll
                for (int j = 0; j < kGKB / 8; ++j) {   // K = 8 TF32 values = 32 bytes per instruction
                    const uint64_t a0 = sw128_desc(base + 0 * kGBlockBytes + 32 * j);
                    const uint64_t a1 = sw128_desc(base + 1 * kGBlockBytes + 32 * j);
                    const uint64_t at = sw128_desc(base + 2 * kGBlockBytes + 32 * j);
                    const uint64_t b0 = sw128_desc(base + 3 * kGBlockBytes + 32 * j);
                    const uint64_t b1 = sw128_desc(base + 4 * kGBlockBytes + 32 * j);
                    const uint64_t bt = sw128_desc(base + 5 * kGBlockBytes + 32 * j);
                    const uint32_t acc = (first && j == 0) ? 0u : 1u;
                    mma_tf32(tmem + 0 * kGM, a0, b0, kIdescTF32, acc);   // level 0
                    mma_tf32(tmem + 1 * kGM, a0, b1, kIdescTF32, acc);   // level 1
                    mma_tf32(tmem + 1 * kGM, a1, b0, kIdescTF32, 1);
                    mma_tf32(tmem + 2 * kGM, a0, bt, kIdescTF32, acc);   // level 2
                    mma_tf32(tmem + 2 * kGM, at, b0, kIdescTF32, 1);
                    mma_tf32(tmem + 2 * kGM, a1, b1, kIdescTF32, 1);
                    mma_tf32(tmem + 3 * kGM, a1, bt, kIdescTF32, acc);   // level 3
                    mma_tf32(tmem + 3 * kGM, at, b1, kIdescTF32, 1);
                }
                mma_commit(&empty[s]);   // stage s may be refilled once these MMAs are done
                if ((k % kGDrain) == kGDrain - 1 || k == nkb - 1) mma_commit(&tfull);
            }
        }
        __syncwarp();
    } else {
        // warps 0-7: row 32 (w mod 4) + lane, columns 64 (w / 4) ... 64 (w / 4) + 63
        constexpr int kCols = kGM / 2;
        float S[kCols], E[kCols];
#pragma unroll
        for (int c = 0; c < kCols; ++c) S[c] = E[c] = 0.f;
        bool ok = true;
        const uint32_t taddr = tmem + (uint32_t(32 * (warp & 3)) << 16) + uint32_t(kCols * (warp >> 2));
        for (int g = 0; g < ngroups; ++g) {
            ok = __all_sync(0xffffffffu, wait_bar(&tfull, g & 1, ctl, tmo));
            if (!ok) break;
            tc_fence_after();
#pragma unroll
            for (int c0 = 0; c0 < kCols; c0 += 8) {
                float v0[8], v1[8];
                tmem_ld8x2(taddr + 0 * kGM + c0, taddr + 1 * kGM + c0, v0, v1);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    float hi, lo, s, e;
                    two_sum(v0[q], __fmul_rn(v1[q], 0x1p-7f), hi, lo);   // exact integers: exact sum
                    two_sum(S[c0 + q], hi, s, e);
                    S[c0 + q] = s;
                    E[c0 + q] = __fadd_rn(E[c0 + q], __fadd_rn(e, lo));
                }
                tmem_ld8x2(taddr + 2 * kGM + c0, taddr + 3 * kGM + c0, v0, v1);
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    E[c0 + q] = __fadd_rn(E[c0 + q], __fmaf_rn(v1[q], 0x1p-21f, __fmul_rn(v0[q], 0x1p-14f)));
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty);
        }
        if (ok && nkb > 0) {
            const int row = 32 * (warp & 3) + lane;
            float2* dst = partial + ((size_t(split) * (size_t(nt) * (nt + 1) / 2) + tile) * kGM + row) * kGM +
                          kCols * (warp >> 2);
#pragma unroll
            for (int c = 0; c < kCols; c += 2)
                reinterpret_cast<float4*>(dst + c)[0] = make_float4(S[c], E[c], S[c + 1], E[c + 1]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kGTmemCols);
    }
}

// Sum the split partial tiles in split order (FP64), scale by 2^(e_i + e_j - 14) / (n - 1),
// write Sigma and Sigma0 (both triangles) with a unit diagonal.
__global__ void k_gram_tc_reduce(Fit f, const float2* __restrict__ partial, const int* __restrict__ expo, int nt,
                                 int nsplit) {
    const int tile = blockIdx.y;
    int bi = 0, rem = tile;
    while (rem >= nt - bi) {
        rem -= nt - bi;
        ++bi;
    }
    const int bj = bi + rem;
    const size_t ntri = size_t(nt) * (nt + 1) / 2;
    const double inv = 1.0 / double(f.n - 1);
    const int p = f.p;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kGM * kGM; e += gridDim.x * blockDim.x) {
        const int r = e / kGM, c = e % kGM;
        const int i = bi * kGM + r, j = bj * kGM + c;
        if (i >= p || j >= p || i > j) continue;
        // split order; eight loads in flight at a time
        double s = 0.0;
        int sp = 0;
        for (; sp + 8 <= nsplit; sp += 8) {
            float2 v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = partial[((size_t(sp + q) * ntri + tile) * kGM + r) * kGM + c];
#pragma unroll
            for (int q = 0; q < 8; ++q) s += double(v[q].x) + double(v[q].y);
        }
        for (; sp < nsplit; ++sp) {
            const float2 v = partial[((size_t(sp) * ntri + tile) * kGM + r) * kGM + c];
            s += double(v.x) + double(v.y);
        }
        const double v = (i == j) ? 1.0 : ldexp(s, expo[i] + expo[j] - 14) * inv;
        f.sig[size_t(i) * p + j] = v;
        f.sig[size_t(j) * p + i] = v;
        f.sig0[size_t(i) * p + j] = v;
        f.sig0[size_t(j) * p + i] = v;
        const float2 vf = sig_pair_f(v);
        f.sigf[size_t(i) * p + j] = vf;
        f.sigf[size_t(j) * p + i] = vf;
    }
}

// ------------------------------------------------------------------ host side
// Split of the sample axis: as many splits as fit the triangle's tiles into one
// wave over the 152 SMs (one CTA per SM), at most 32, every split at least one k-step.
struct GramTcPlan {
    int nt, ntri, kb_total, kb_per_split, nsplit;
};
static GramTcPlan gram_tc_plan(long long p, int ld) {
    GramTcPlan g;
    g.nt = int((p + kGM - 1) / kGM);
    g.ntri = g.nt * (g.nt + 1) / 2;
    g.kb_total = ld / kGKB;
    int want = 152 / g.ntri;
    want = want < 1 ? 1 : (want > 32 ? 32 : want);
    if (want > g.kb_total) want = g.kb_total;
    g.kb_per_split = (g.kb_total + want - 1) / want;
    g.nsplit = (g.kb_total + g.kb_per_split - 1) / g.kb_per_split;
    return g;
}

size_t gram_tc_partial_bytes(long long p, int ld) {
    const GramTcPlan g = gram_tc_plan(p, ld);
    return size_t(g.nsplit) * size_t(g.ntri) * kGM * kGM * sizeof(float2);
}

size_t gram_tc_digit_bytes(long long p, int ld) {
    return 3 * size_t(p) * size_t(ld) * sizeof(float) + size_t(p) * sizeof(int);
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry-point query, so the
// library needs no link against the driver library.
static EncodeTiledFn encode_fn() {
    static const EncodeTiledFn fn = [] {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return EncodeTiledFn(nullptr);
        }
        return reinterpret_cast<EncodeTiledFn>(ptr);
    }();
    return fn;
}

// 2-D map over a p x ld FP32 matrix (row stride ld), boxes of 32 samples x 128 rows,
// 128-byte swizzle, rows beyond p read as zero.
static bool make_map(CUtensorMap* map, void* base, int p, int ld) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {cuuint64_t(ld), cuuint64_t(p)};
    const cuuint64_t strides[1] = {cuuint64_t(ld) * sizeof(float)};
    const cuuint32_t box[2] = {cuuint32_t(kGKB), cuuint32_t(kGM)};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_gram_tc(const Fit& f, void* digits, void* partial, cudaStream_t st) {
    const size_t plane = size_t(f.p) * f.ld;
    float* d0 = static_cast<float*>(digits);
    float* d1 = d0 + plane;
    float* tt = d1 + plane;
    int* expo = reinterpret_cast<int*>(tt + plane);
    k_digits<<<f.p, kDigitThreads, 0, st>>>(static_cast<const float*>(f.xt), d0, d1, tt, expo, f.ld);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    GramMaps maps;
    if (!make_map(&maps.d0, d0, f.p, f.ld) || !make_map(&maps.d1, d1, f.p, f.ld) || !make_map(&maps.tt, tt, f.p, f.ld))
        return cudaErrorInvalidValue;
    const GramTcPlan g = gram_tc_plan(f.p, f.ld);
    e = ensure_smem_attr(reinterpret_cast<const void*>(k_gram_tc), gram_tc_smem_bytes());
    if (e != cudaSuccess) return e;
    float2* part = static_cast<float2*>(partial);
    k_gram_tc<<<g.ntri * g.nsplit, kGThreads, gram_tc_smem_bytes(), st>>>(maps, part, g.nt, g.kb_per_split,
                                                                         g.kb_total, g.nsplit, f.ctl);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_gram_tc_reduce<<<dim3(16, g.ntri), 256, 0, st>>>(f, part, expo, g.nt, g.nsplit);
    return cudaGetLastError();
}

}  // namespace lingam

// k_gram.cu -- CalculateCovMat (Algorithm 3): Sigma = Xn Xn^T / (n-1)
// of the normalised rows, the covariance the closed forms of Sec. III-E start
// from.  SIMT version: 64 x 64 output tiles of the upper triangle, K-chunks of
// 32 samples staged in shared memory; FP32 products with FP32 chunk sums
// folded into Kahan-compensated FP32 totals (mixed path), or FP64 throughout.
// The diagonal is exactly 1 (normalised rows).
#include <type_traits>

#include "common.cuh"
#include "launch.h"

namespace lingam {

constexpr int kGT = 64;   // output tile
constexpr int kGK = 32;   // samples per chunk

template <class T>
__global__ void __launch_bounds__(256) k_gram(Fit f) {
    __shared__ __align__(16) T As[kGK][kGT + 4];
    __shared__ __align__(16) T Bs[kGK][kGT + 4];
    const int p = f.p, ld = f.ld, tid = threadIdx.x;
    // blockIdx.x -> (bi, bj) with bi <= bj
    const int nt = (p + kGT - 1) / kGT;
    int rem = blockIdx.x, bi = 0;
    while (rem >= nt - bi) {
        rem -= nt - bi;
        ++bi;
    }
    const int bj = bi + rem;
    const int i0 = bi * kGT, j0 = bj * kGT;
    const T* xt = static_cast<const T*>(f.xt);
    const int ty = tid >> 4, tx = tid & 15;

    T sum[4][4], comp[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            sum[a][b] = T(0);
            comp[a][b] = T(0);
        }
    for (int k0 = 0; k0 < ld; k0 += kGK) {
        // stage: 64 rows x 32 samples of each operand, transposed to [k][row]
        for (int e = tid; e < kGT * kGK; e += 256) {
            const int rr = e / kGK, kk = e % kGK;
            const int gi = i0 + rr, gj = j0 + rr;
            As[kk][rr] = gi < p ? xt[size_t(gi) * ld + k0 + kk] : T(0);
            Bs[kk][rr] = gj < p ? xt[size_t(gj) * ld + k0 + kk] : T(0);
        }
        __syncthreads();
        T acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
#pragma unroll 8
        for (int kk = 0; kk < kGK; ++kk) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][ty * 4 + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx * 4 + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                if constexpr (std::is_same<T, float>::value) {   // Kahan step
                    const float y = acc[a][b] - comp[a][b];
                    const float t = sum[a][b] + y;
                    comp[a][b] = (t - sum[a][b]) - y;
                    sum[a][b] = t;
                } else {
                    sum[a][b] += acc[a][b];
                }
            }
        __syncthreads();
    }
    const double scale = 1.0 / double(f.n - 1);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = i0 + ty * 4 + a, j = j0 + tx * 4 + b;
            if (i < p && j < p && i <= j) {
                const double v = (i == j) ? 1.0 : double(sum[a][b]) * scale;
                f.sig[size_t(i) * p + j] = v;
                f.sig[size_t(j) * p + i] = v;
                f.sig0[size_t(i) * p + j] = v;
                f.sig0[size_t(j) * p + i] = v;
            }
        }
}

cudaError_t launch_gram(const Fit& f, cudaStream_t st) {
    const int nt = (f.p + kGT - 1) / kGT;
    const int grid = nt * (nt + 1) / 2;
    if (f.precision == LINGAM_MIXED) k_gram<float><<<grid, 256, 0, st>>>(f);
    else k_gram<double><<<grid, 256, 0, st>>>(f);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ small problems of a batch
// CalculateCovMat of every problem of a batch table with p <= kSmallGramP and rows of at most
// kSmallGramLd samples (mixed path) in one launch, where the per-problem tensor-core Gram
// would pay three launches and their fixed costs per problem.  A CTA takes 256 elements of
// one problem's upper triangle, one per thread, in the order t = j (j + 1) / 2 + i (i <= j),
// so that a warp's threads read consecutive rows of the staged chunk; every chunk of kSGK
// samples of all the problem's rows is staged in shared memory.  Each product of two FP32
// row values is split exactly into hi + lo (TwoProd by fma) and added into a float-float
// sum, so the result is the exact Gram of the FP32 rows up to the float-float rounding, like
// the tensor-core version's.
constexpr int kSGOut = 256;
constexpr int kSGK = 32;

__host__ __device__ inline int small_gram_units(long long p, long long ld) {
    if (p < 1 || p > kSmallGramP || ld > kSmallGramLd) return 0;
    const long long tri = p * (p + 1) / 2;
    return int((tri + kSGOut - 1) / kSGOut);
}

__device__ __forceinline__ void ff_mac(float a, float b, float& hi, float& lo) {
    const float pr = a * b, pe = fmaf(a, b, -pr);   // a b = pr + pe exactly
    const float s = hi + pr, bb = s - hi;
    lo += ((hi - (s - bb)) + (pr - bb)) + pe;        // TwoSum error of hi + pr
    hi = s;
}

__global__ void __launch_bounds__(kSGOut) k_gram_small_batch(const Fit* __restrict__ fits, int count) {
    constexpr int NW = kSGOut / 32;
    __shared__ int s_off[kBatchLaunchMax + 1];
    __shared__ int s_wsum[NW];
    __shared__ float xs[kSGK][kSmallGramP + 1];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    // the problems' first units (an exclusive prefix over the table, count <= kBatchLaunchMax)
    int run = 0;
    for (int base = 0; base < count; base += kSGOut) {
        const int d = base + tid;
        const int u = d < count ? small_gram_units(fits[d].p, fits[d].ld) : 0;
        int x = u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_wsum[wid] = x;
        __syncthreads();
        int wo = 0, tot = 0;
        for (int w = 0; w < NW; ++w) {
            wo += w < wid ? s_wsum[w] : 0;
            tot += s_wsum[w];
        }
        if (d < count) s_off[d] = run + wo + x - u;
        run += tot;
        __syncthreads();
    }
    if (tid == 0) s_off[count] = run;
    __syncthreads();
    const int b = int(blockIdx.x);
    if (b >= s_off[count]) return;   // the whole CTA
    int d = 0, hi_d = count - 1;     // the last problem whose first unit is at most b
    while (d < hi_d) {
        const int mid = (d + hi_d + 1) >> 1;
        if (s_off[mid] <= b) d = mid;
        else hi_d = mid - 1;
    }
    const Fit& f = fits[d];
    const int p = f.p, ld = f.ld;
    const int t = (b - s_off[d]) * kSGOut + tid;
    const bool mine = t < p * (p + 1) / 2;
    int j = 0, i = 0;
    if (mine) {
        j = int((sqrtf(8.f * float(t) + 1.f) - 1.f) * 0.5f);
        while (j * (j + 1) / 2 > t) --j;
        while ((j + 1) * (j + 2) / 2 <= t) ++j;
        i = t - j * (j + 1) / 2;
    }
    float shi = 0.f, slo = 0.f;
    const float* xt = static_cast<const float*>(f.xt);
    const int nst = p * kSGK;
    for (int k0 = 0; k0 < ld; k0 += kSGK) {
        __syncthreads();   // the previous chunk is consumed
        for (int e = tid; e < nst; e += kSGOut) {
            const int r = e >> 5, kk = e & (kSGK - 1);
            xs[kk][r] = xt[size_t(r) * ld + k0 + kk];
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < kSGK; ++kk) ff_mac(xs[kk][i], xs[kk][j], shi, slo);
    }
    if (!mine) return;
    const double v = i == j ? 1.0 : (double(shi) + double(slo)) / double(f.n - 1);
    f.sig[size_t(i) * p + j] = v;
    f.sig[size_t(j) * p + i] = v;
    f.sig0[size_t(i) * p + j] = v;
    f.sig0[size_t(j) * p + i] = v;
    const float2 vf = sig_pair_f(v);
    f.sigf[size_t(i) * p + j] = vf;
    f.sigf[size_t(j) * p + i] = vf;
}

int gram_small_batch_units(const long long* p, const int* ld, int count) {
    int u = 0;
    for (int k = 0; k < count; ++k) u += small_gram_units(p[k], ld[k]);
    return u;
}

cudaError_t launch_gram_small_batch(const Fit* fits_dev, int count, int units, cudaStream_t st) {
    if (count < 1 || count > kBatchLaunchMax || units < 1) return cudaErrorInvalidValue;
    k_gram_small_batch<<<units, kSGOut, 0, st>>>(fits_dev, count);
    return cudaGetLastError();
}

}  // namespace lingam

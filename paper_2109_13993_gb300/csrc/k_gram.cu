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

}  // namespace lingam

// k_rows.cu -- NormalizeData (Algorithm 3): per-row normalisation of
// the input with the first H(x) terms.
#include <type_traits>

#include "common.cuh"
#include "launch.h"

namespace lingam {

constexpr int kRowThreads = 256;

// ------------------------------------------------------------------ NormalizeData
// One CTA per row: mean, standard deviation with divisor n-1 (both FP64), the
// padded normalised row (zeros beyond n) and H(x) - H(nu).  Sample t of the row is
// xr[t], or xr[idx[t]] when idx is given (a bootstrap resample of the columns).
template <class Tin, class T>
__device__ void standardize_row(const Fit& f, const Tin* __restrict__ xr, const int* __restrict__ idx, int row,
                                double* red) {
    const int n = f.n, ld = f.ld, tid = threadIdx.x;
    auto at = [&](int t) { return double(idx ? xr[idx[t]] : xr[t]); };
    double s = 0.0;
    bool finite = true;
    for (int t = tid; t < n; t += kRowThreads) {
        const double v = at(t);
        finite &= isfinite(v);
        s += v;
    }
    if (__syncthreads_or(!finite)) {
        if (tid == 0) set_status(f.ctl, LINGAM_EDEGENERATE);
        return;
    }
    const double mu = block_sum(s, red) / double(n);
    double q = 0.0;
    for (int t = tid; t < n; t += kRowThreads) {
        const double d = at(t) - mu;
        q = fma(d, d, q);
    }
    const double var = block_sum(q, red) / double(n - 1);
    if (!(var > 0.0) || !isfinite(var)) {
        if (tid == 0) set_status(f.ctl, LINGAM_EDEGENERATE);
        return;
    }
    const double sd = sqrt(var), inv = 1.0 / sd;
    T* out = static_cast<T*>(f.xt) + size_t(row) * ld;
    T lcc = T(0), g = T(0);
    for (int t = tid; t < ld; t += kRowThreads) {
        T u = T(0);
        if (t < n) {
            u = T((at(t) - mu) * inv);
            mom_add(u, lcc, g);
        }
        out[t] = u;
    }
    const double L = block_sum(double(lcc), red), G = block_sum(double(g), red);
    if (tid == 0) {
        f.mu[row] = mu;
        f.sd[row] = sd;
        f.hx[row] = hterm(L, G, double(n));
        f.vstat[row] = var_stats(L, G, n, ld);
        f.flags[row] = kAlive;
    }
}

template <class Tin, class T>
__global__ void __launch_bounds__(kRowThreads) k_standardize(Fit f, const Tin* __restrict__ x) {
    __shared__ double red[kRowThreads / 32];
    standardize_row<Tin, T>(f, x + size_t(blockIdx.x) * f.n, nullptr, blockIdx.x, red);
}

// All rows of many problems: CTA g takes row g - rowoff[d] of the problem d with
// rowoff[d] <= g < rowoff[d + 1].
template <class Tin, class T>
__global__ void __launch_bounds__(kRowThreads) k_standardize_batch(const Fit* __restrict__ fits,
                                                                 const SrcDesc* __restrict__ src,
                                                                 const int* __restrict__ rowoff, int count) {
    __shared__ double red[kRowThreads / 32];
    const int g = blockIdx.x;
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (rowoff[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    const Fit f = fits[lo];
    if (((volatile Ctl*)f.ctl)->status != 0) return;
    const int row = g - rowoff[lo];
    const SrcDesc sd = src[lo];
    standardize_row<Tin, T>(f, static_cast<const Tin*>(sd.x) + size_t(row) * sd.ld, sd.idx, row, red);
}

// Per-problem start of a batch: orders unset, tile counters and report arrays zero.
__global__ void k_batch_init(const Fit* __restrict__ fits, int count) {
    const Fit f = fits[blockIdx.x];
    for (int k = threadIdx.x; k < f.p; k += blockDim.x) {
        f.order[k] = -1;
        f.rep_pairs[k] = 0;
        f.rep_root_score[k] = 0.0;
        f.rep_margin[k] = 0.0;
    }
    for (int t = threadIdx.x; t < f.maxtiles; t += blockDim.x) f.tile_cnt[t] = 0;
}

cudaError_t launch_standardize_batch(const Fit* fits, const SrcDesc* src, const int* rowoff, int count, int rows,
                                     int precision, int input_dtype, cudaStream_t st) {
    k_batch_init<<<count, 256, 0, st>>>(fits, count);
    if (precision == LINGAM_MIXED) {
        if (input_dtype == LINGAM_F32) k_standardize_batch<float, float><<<rows, kRowThreads, 0, st>>>(fits, src, rowoff, count);
        else k_standardize_batch<double, float><<<rows, kRowThreads, 0, st>>>(fits, src, rowoff, count);
    } else {
        if (input_dtype == LINGAM_F32) k_standardize_batch<float, double><<<rows, kRowThreads, 0, st>>>(fits, src, rowoff, count);
        else k_standardize_batch<double, double><<<rows, kRowThreads, 0, st>>>(fits, src, rowoff, count);
    }
    return cudaGetLastError();
}

cudaError_t launch_standardize(const Fit& f, const void* x, int input_dtype, cudaStream_t st) {
    if (f.precision == LINGAM_MIXED) {
        if (input_dtype == LINGAM_F32)
            k_standardize<float, float><<<f.p, kRowThreads, 0, st>>>(f, static_cast<const float*>(x));
        else
            k_standardize<double, float><<<f.p, kRowThreads, 0, st>>>(f, static_cast<const double*>(x));
    } else {
        if (input_dtype == LINGAM_F32)
            k_standardize<float, double><<<f.p, kRowThreads, 0, st>>>(f, static_cast<const float*>(x));
        else
            k_standardize<double, double><<<f.p, kRowThreads, 0, st>>>(f, static_cast<const double*>(x));
    }
    return cudaGetLastError();
}

}  // namespace lingam

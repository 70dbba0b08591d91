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
// The FP32 working copy (mixed path) in float-float arithmetic: FP64 operations are slow on
// this part, and float-float sums keep about 48 bits.  The sum of the samples and the sum of
// the squared deviations are float-float (a sample of an FP64 input enters as its
// float-float split; a deviation v - mu is formed exactly by TwoSum and its square by
// TwoProd); mean, variance and 1/sd are formed once per row in FP64.  The normalised sample
// is the float-float deviation times 1/sd (float-float), rounded once to FP32.
__device__ __forceinline__ float2 ff_of(float v) { return make_float2(v, 0.f); }
__device__ __forceinline__ float2 ff_of(double v) {
    const float hi = float(v);
    return make_float2(hi, float(v - double(hi)));
}
// a - (mh + ml) as float-float
__device__ __forceinline__ float2 ff_dev(float2 a, float mh, float ml) {
    return ff_add(a, make_float2(-mh, -ml));
}
// Fixed-order float-float block sum; the result to every thread.
__device__ __forceinline__ float2 block_ff_sum(float2 v, float2* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = ff_add(v, make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o)));
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    float2 s = red[0];
    for (int w = 1; w < kRowThreads / 32; ++w) s = ff_add(s, red[w]);
    return s;
}

// Returns false (before any write) when the row's largest magnitude lies outside
// [2^-60, 2^60]: there the float-float sums could overflow or lose their low parts, and the
// caller takes the FP64 routine.
template <class Tin>
__device__ bool standardize_row_ff(const Fit& f, const Tin* __restrict__ xr, const int* __restrict__ idx, int row,
                                   float2* red, double* bc) {
    const int n = f.n, ld = f.ld, tid = threadIdx.x;
    auto at = [&](int t) { return idx ? xr[idx[t]] : xr[t]; };
    float2 s = make_float2(0.f, 0.f);
    float amax = 0.f;
    bool finite = true;
    for (int t = tid; t < n; t += kRowThreads) {
        const Tin v = at(t);
        finite &= isfinite(v);
        s = ff_add(s, ff_of(v));
        amax = fmaxf(amax, fabsf(float(v)));
    }
    if (__syncthreads_or(!finite)) {
        if (tid == 0) set_status(f.ctl, LINGAM_EDEGENERATE);
        return true;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if ((tid & 31) == 0) red[tid >> 5].x = amax;
    __syncthreads();
    amax = red[0].x;
    for (int w = 1; w < kRowThreads / 32; ++w) amax = fmaxf(amax, red[w].x);
    if (!(amax >= 0x1p-60f && amax <= 0x1p60f)) return false;   // the same for every thread
    s = block_ff_sum(s, red);
    if (tid == 0) bc[0] = (double(s.x) + double(s.y)) / double(n);
    __syncthreads();
    const double mu = bc[0];
    const float mh = float(mu), ml = float(mu - double(mh));
    // the deviations scaled by 2^-e (exactly), |v| < 2^(e+1), so that their squares stay in range
    const int e = ilogbf(amax);
    const float sc = ldexpf(1.f, -e);
    float2 q = make_float2(0.f, 0.f);
    for (int t = tid; t < n; t += kRowThreads) {
        float2 d = ff_dev(ff_of(at(t)), mh, ml);
        d.x *= sc;
        d.y *= sc;
        const float sq = d.x * d.x;
        q = ff_add(q, make_float2(sq, fmaf(d.x, d.x, -sq) + 2.f * d.x * d.y));
    }
    q = block_ff_sum(q, red);
    if (tid == 0) {
        const double var = ldexp(double(q.x) + double(q.y), 2 * e) / double(n - 1);
        bc[1] = var;
        bc[2] = 1.0 / sqrt(var);
    }
    __syncthreads();
    const double var = bc[1];
    if (!(var > 0.0) || !isfinite(var)) {
        if (tid == 0) set_status(f.ctl, LINGAM_EDEGENERATE);
        return true;
    }
    // 1/sd as float-float, so that a row is not scaled by the FP32 rounding of 1/sd
    const float ih = float(bc[2]), il = float(bc[2] - double(ih));
    float* out = static_cast<float*>(f.xt) + size_t(row) * ld;
    float lcc = 0.f, g = 0.f;
    for (int t = tid; t < ld; t += kRowThreads) {
        float u = 0.f;
        if (t < n) {
            const float2 d = ff_dev(ff_of(at(t)), mh, ml);
            u = fmaf(d.x, ih, fmaf(d.x, il, d.y * ih));
            mom_add(u, lcc, g);
        }
        out[t] = u;
    }
    const float2 L = block_ff_sum(make_float2(lcc, 0.f), red);
    const float2 G = block_ff_sum(make_float2(g, 0.f), red);
    if (tid == 0) {
        const double Ld = double(L.x) + double(L.y), Gd = double(G.x) + double(G.y);
        f.mu[row] = mu;
        f.sd[row] = sqrt(var);
        f.hx[row] = hterm_inv(Ld, Gd, f.inv_n);
        f.vstat[row] = var_stats_inv(Ld, Gd, n, ld, f.inv_n);
        f.flags[row] = kAlive;
    }
    return true;
}

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

// One row of the working copy: float-float arithmetic for an FP32 copy (FP64 for a row whose
// magnitudes leave [2^-60, 2^60]), FP64 for an FP64 one.
template <class Tin, class T>
__device__ __forceinline__ void normalise_row(const Fit& f, const Tin* __restrict__ xr, const int* __restrict__ idx,
                                              int row) {
    __shared__ double red[kRowThreads / 32];
    if constexpr (std::is_same<T, float>::value) {
        __shared__ float2 red2[kRowThreads / 32];
        __shared__ double bc[3];
        if (standardize_row_ff<Tin>(f, xr, idx, row, red2, bc)) return;
        __syncthreads();   // red2 is not reused, but keep the fallback's start ordered
    }
    standardize_row<Tin, T>(f, xr, idx, row, red);
}

template <class Tin, class T>
__global__ void __launch_bounds__(kRowThreads) k_standardize(Fit f, const Tin* __restrict__ x) {
    normalise_row<Tin, T>(f, x + size_t(blockIdx.x) * f.n, nullptr, blockIdx.x);
}

// All rows of many problems: CTA g takes row g - rowoff[d] of the problem d with
// rowoff[d] <= g < rowoff[d + 1].
template <class Tin, class T>
__global__ void __launch_bounds__(kRowThreads) k_standardize_batch(const Fit* __restrict__ fits,
                                                                 const SrcDesc* __restrict__ src,
                                                                 const int* __restrict__ rowoff, int count) {
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
    normalise_row<Tin, T>(f, static_cast<const Tin*>(sd.x) + size_t(row) * sd.ld, sd.idx, row);
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

// k_rows.cu -- NormalizeData (Algorithm 3): per-row normalisation of
// the input with the first H(x) terms.
#include <type_traits>

#include "common.cuh"
#include "launch.h"

namespace lingam {

constexpr int kRowThreads = 256;

// ------------------------------------------------------------------ NormalizeData
// One CTA per row: mean, standard deviation with divisor n-1 (both FP64), the
// padded normalised row (zeros beyond n) and H(x) - H(nu).
template <class Tin, class T>
__global__ void __launch_bounds__(kRowThreads) k_standardize(Fit f, const Tin* __restrict__ x) {
    __shared__ double red[kRowThreads / 32];
    const int row = blockIdx.x, n = f.n, ld = f.ld, tid = threadIdx.x;
    const Tin* xr = x + size_t(row) * n;
    double s = 0.0;
    bool finite = true;
    for (int t = tid; t < n; t += kRowThreads) {
        const double v = double(xr[t]);
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
        const double d = double(xr[t]) - mu;
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
            u = T((double(xr[t]) - mu) * inv);
            mom_add(u, lcc, g);
        }
        out[t] = u;
    }
    const double L = block_sum(double(lcc), red), G = block_sum(double(g), red);
    if (tid == 0) {
        f.mu[row] = mu;
        f.sd[row] = sd;
        f.hx[row] = hterm(L, G, double(n));
        f.flags[row] = kAlive;
    }
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

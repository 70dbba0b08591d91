// k_rows.cu -- per-row kernels of the ordering loop (Algorithm 3):
//   NormalizeData (line 3), the start of an iteration (candidate order, first
//   wave), UpdateData (Algorithm 7) fused with the new H(x_w) terms, and
//   UpdateCovMat (Algorithm 8 / Eq. CovUpdate).
#include <type_traits>

#include "common.cuh"
#include "launch.h"

namespace lingam {

constexpr int kRowThreads = 256;

// Sum over one thread's samples of (log cosh u - beta) and u e^{-u^2/2} for a
// normalised sample u (Eq. HApp), FP32 on the SFU:
//   log cosh u = |u| + ln2 * log2(1 + 2^{-2 log2(e) |u|}) - ln 2.
struct Mom {
    double lcc, g;
};
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

// ------------------------------------------------------------------ start of an iteration
// One CTA.  Candidate order sigma = the variables of U sorted by the previous
// iteration's scores (iteration 0: by H(x) - H(nu), most non-Gaussian first),
// lowest index on ties; the first wave's columns are the first kTJ of them.
constexpr int kPlanThreads = 1024;
constexpr int kSortMax = 8192;

__global__ void __launch_bounds__(kPlanThreads) k_plan(Fit f, int it, int nsplit) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int red[kPlanThreads / 32];
    Ctl* ctl = f.ctl;
    const int p = f.p, tid = threadIdx.x;
    // U in index order
    int r = 0;
    for (int base = 0; base < p; base += kPlanThreads) {
        const int v = base + tid;
        const int a = (v < p) ? (f.flags[v] & kAlive) : 0;
        int tot;
        const int rank = r + block_scan01(a ? 1 : 0, red, &tot);
        if (a) f.sigma[rank] = v;
        r += tot;
        __syncthreads();
    }
    // sort by key (bitonic, in shared memory) when U is small enough
    if (r <= kSortMax && r > 1) {
        int N = 1;
        while (N < r) N <<= 1;
        double* key = reinterpret_cast<double*>(sm);
        int* idx = reinterpret_cast<int*>(key + kSortMax);
        for (int k = tid; k < N; k += kPlanThreads) {
            if (k < r) {
                const int v = f.sigma[k];
                key[k] = it == 0 ? f.hx[v] : f.prev[v];
                idx[k] = v;
            } else {
                key[k] = INFINITY;
                idx[k] = 0x7fffffff;
            }
        }
        __syncthreads();
        for (int size = 2; size <= N; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int k = tid; k < N; k += kPlanThreads) {
                    const int l = k ^ stride;
                    if (l > k) {
                        const bool up = (k & size) == 0;
                        const bool gt = key[k] > key[l] || (key[k] == key[l] && idx[k] > idx[l]);
                        if (gt == up) {
                            const double tk = key[k];
                            key[k] = key[l];
                            key[l] = tk;
                            const int ti = idx[k];
                            idx[k] = idx[l];
                            idx[l] = ti;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int k = tid; k < r; k += kPlanThreads) f.sigma[k] = idx[k];
        __syncthreads();
    }
    // reset per-iteration state
    for (int k = tid; k < r; k += kPlanThreads) {
        const int v = f.sigma[k];
        f.part[v] = 0.0;
        f.flags[v] = kAlive;
        f.rows[k] = v;
    }
    if (f.want_scores)
        for (int v = tid; v < p; v += kPlanThreads) f.rep_scores[size_t(it) * p + v] = NAN;
    __syncthreads();
    if (tid == 0) {
        ctl->it = it;
        ctl->r = r;
        ctl->wave = 0;
        ctl->wave_ctas_done = 0;
        ctl->best = INFINITY;
        ctl->best_var = -1;
        ctl->pairs_it = 0;
        ctl->nsplit = nsplit;
        if (r <= 1) {
            // Algorithm 2, lines 1-3: a single variable is the root
            const int root = r == 1 ? f.sigma[0] : -1;
            ctl->root = root;
            ctl->done = 1;
            if (root >= 0) {
                f.order[it] = root;
                if (f.want_scores) f.rep_scores[size_t(it) * p + root] = 0.0;
            }
            f.rep_root_score[it] = 0.0;
            f.rep_margin[it] = INFINITY;
            f.rep_pairs[it] = 0;
            ctl->ncol = 0;
            ctl->nrow = 0;
            ctl->ntiles = 0;
        } else {
            ctl->done = 0;
            const int nc = r < kTJ ? r : kTJ;
            for (int c = 0; c < nc; ++c) f.cols[c] = f.sigma[c];
            ctl->ncol = nc;
            ctl->nrow = r;
            ctl->ntiles = (r + kTI - 1) / kTI;
        }
    }
}

cudaError_t launch_plan(const Fit& f, int it, int nsplit, cudaStream_t st) {
    const size_t smem = size_t(kSortMax) * (sizeof(double) + sizeof(int));
    cudaError_t e = ensure_smem_attr(reinterpret_cast<const void*>(k_plan), smem);
    if (e != cudaSuccess) return e;
    k_plan<<<1, kPlanThreads, smem, st>>>(f, it, nsplit);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ UpdateData (Algorithm 7)
// CTA b handles variable w = sigma[b] of the iteration that just chose its root:
//   x_w <- (x_w - Sigma[w,root] x_root) / sqrt(1 - Sigma[w,root]^2),
// then recomputes H(x_w) - H(nu).  The root itself is marked removed.  Each
// variable's score is kept as the next iteration's candidate key.
template <class T>
__global__ void __launch_bounds__(kRowThreads) k_remove_root_data(Fit f, int it, int r) {
    __shared__ double red[kRowThreads / 32];
    Ctl* ctl = f.ctl;
    const int b = blockIdx.x, tid = threadIdx.x, p = f.p, ld = f.ld;
    const int root = ctl->root;
    if (root < 0) return;
    const int w = f.sigma[b];
    if (tid == 0) f.prev[w] = f.part[w];
    if (w == root) {
        if (tid == 0) {
            f.flags[w] = 0;
            f.inv_root[w] = 0.0;
        }
        return;
    }
    const double c = f.sig[size_t(w) * p + root];
    const double om = fma(-c, c, 1.0);
    if (!(om > 1e-14)) {
        if (tid == 0) set_status(ctl, LINGAM_EDEGENERATE);
        return;
    }
    const double inv = 1.0 / sqrt(om);
    if (tid == 0) f.inv_root[w] = inv;
    T* xw = static_cast<T*>(f.xt) + size_t(w) * ld;
    const T* xr = static_cast<const T*>(f.xt) + size_t(root) * ld;
    const T cc = T(c), ii = T(inv);
    T lcc = T(0), g = T(0);
    for (int t = tid; t < ld; t += kRowThreads) {
        T u;
        if constexpr (std::is_same<T, float>::value) u = fmaf(-cc, xr[t], xw[t]) * ii;
        else u = fma(-cc, xr[t], xw[t]) * ii;
        xw[t] = u;
        if (t < f.n) mom_add(u, lcc, g);
    }
    const double L = block_sum(double(lcc), red), G = block_sum(double(g), red);
    if (tid == 0) f.hx[w] = hterm(L, G, double(f.n));
}

// ------------------------------------------------------------------ UpdateCovMat (Algorithm 8)
// Eq. CovUpdate on the normalised rows, for w, j in U without the root:
//   Sigma[w,j] <- (Sigma[w,j] - Sigma[w,root] Sigma[j,root]) / (sqrt(1-Sigma[w,root]^2) sqrt(1-Sigma[j,root]^2)),
// diagonal kept at 1.  The root's row and column are not written, so the update
// is done in place.  Grid: (ceil(r/32), ceil(r/32)) tiles of sigma positions.
__global__ void __launch_bounds__(256) k_remove_root_cov(Fit f, int r) {
    const int root = f.ctl->root;
    if (root < 0) return;
    const int p = f.p;
    const int a0 = blockIdx.y * 32, b0 = blockIdx.x * 32;
    const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
    const int b = b0 + tx;
    if (b >= r) return;
    const int j = f.sigma[b];
    if (j == root) return;
    const double cj = f.sig[size_t(j) * p + root], ij = f.inv_root[j];
    for (int a = a0 + ty; a < a0 + 32 && a < r; a += 8) {
        const int w = f.sigma[a];
        if (w == root) continue;
        double* s = f.sig + size_t(w) * p + j;
        if (w == j) {
            *s = 1.0;
        } else {
            const double cw = f.sig[size_t(w) * p + root];
            *s = (*s - cw * cj) * (f.inv_root[w] * ij);
        }
    }
}

cudaError_t launch_remove_root(const Fit& f, int it, int r, cudaStream_t st) {
    if (f.precision == LINGAM_MIXED) k_remove_root_data<float><<<r, kRowThreads, 0, st>>>(f, it, r);
    else k_remove_root_data<double><<<r, kRowThreads, 0, st>>>(f, it, r);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 grid((r + 31) / 32, (r + 31) / 32);
    k_remove_root_cov<<<grid, 256, 0, st>>>(f, r);
    return cudaGetLastError();
}

}  // namespace lingam

// k_bfit.cu -- causal strengths B from the causal order (Algorithm 1, last
// line; "conventional covariance-based regression", Sec. II-C), FP64.
//
// B row K[k] holds the least-squares coefficients of x_{K[k]} on its
// predecessors x_{K[0..k-1]}.  With C the covariance of the original variables
// permuted into the order K and C = R R^T its Cholesky factorisation (R lower
// triangular), the innovations e = diag(R) R^{-1} x are uncorrelated and
// x = (I - diag(R) R^{-1}) x + e, so B_K = I - diag(R) R^{-1}, strictly lower
// triangular; B is B_K with rows and columns mapped back to variable indices.
#include <algorithm>

#include "common.cuh"
#include "launch.h"

namespace lingam {

// C[a][b] = sd_{K[a]} sd_{K[b]} Sigma0[K[a]][K[b]]  (original units)
__global__ void k_perm_cov(Fit f) {
    const int p = f.p;
    const int a = blockIdx.y * 16 + (threadIdx.x >> 4), b = blockIdx.x * 16 + (threadIdx.x & 15);
    if (a >= p || b >= p) return;
    const int ia = f.order[a], ib = f.order[b];
    f.cmat[size_t(a) * p + b] = f.sd[ia] * f.sd[ib] * f.sig0[size_t(ia) * p + ib];
}

// Right-looking Cholesky C = R R^T (R lower) in one cooperative launch, as a data flow
// over rows.  The working matrix is the upper triangle U of C (row k of U holds column k
// of C, so every access below is along a row).  At step k, row k of rmat receives
// R[i][k] = U[k][i] / sqrt(U[k][k]) (i >= k) and the rows i > k lose the rank-one term
// U[i][j] -= U[k][i] U[k][j] / U[k][k] (j >= i).  Row i belongs to CTA i mod G for the
// whole factorisation, so its successive updates follow one another inside one CTA;
// step k needs only row k final, which its owner publishes (ready[k] = 1) as soon as
// it has applied step k - 1 to it, before its other rows, so the next steps start while
// the bulk of the current one is still running.  A non-positive pivot records
// LINGAM_EDEGENERATE (every CTA reads the same final pivot, so all leave at the same
// step); every wait is bounded by the fit's timeout.
constexpr int kCholThreads = 256;
constexpr int kCholRows = 128;   // rows of one CTA staged at a time
constexpr int kCholBatch = 8;    // elements per thread with their loads in flight together

// U[i][j] -= a U[k][j] for the rows i0, i0 + G, ... (< p, at most kCholRows of them) and
// j >= i, their elements numbered one after another over the CTA's threads.
__device__ void chol_rows(double* U, const double* uk, double inv, int p, int i0, int G, int* s_i, int* s_off,
                          double* s_a) {
    const int tid = threadIdx.x;
    const int nr = min(kCholRows, (p - 1 - i0) / G + 1);
    __syncthreads();   // the previous row table is no longer read
    for (int r = tid; r < nr; r += kCholThreads) {
        const int i = i0 + r * G;
        s_i[r] = i;
        s_a[r] = __ldcg(uk + i) * inv;
    }
    if (tid == 0) {
        int o = 0;
        for (int r = 0; r < nr; ++r) {
            s_off[r] = o;
            o += p - (i0 + r * G);
        }
        s_off[nr] = o;
    }
    __syncthreads();
    const int tot = s_off[nr];
    for (int base = tid; base < tot; base += kCholBatch * kCholThreads) {
        size_t at[kCholBatch];
        int jj[kCholBatch];
        double av[kCholBatch], x[kCholBatch], y[kCholBatch];
#pragma unroll
        for (int q = 0; q < kCholBatch; ++q) {
            const int idx = base + q * kCholThreads;
            jj[q] = -1;
            if (idx < tot) {
                int lo = 0, hi = nr - 1;   // the row: last r with s_off[r] <= idx
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_off[mid] <= idx) lo = mid;
                    else hi = mid - 1;
                }
                const int i = s_i[lo];
                jj[q] = i + (idx - s_off[lo]);
                at[q] = size_t(i) * p + jj[q];
                av[q] = s_a[lo];
            }
        }
#pragma unroll
        for (int q = 0; q < kCholBatch; ++q)
            if (jj[q] >= 0) {
                x[q] = __ldcg(uk + jj[q]);
                y[q] = __ldcg(U + at[q]);
            }
#pragma unroll
        for (int q = 0; q < kCholBatch; ++q)
            if (jj[q] >= 0) U[at[q]] = fma(-av[q], x[q], y[q]);
    }
}

__global__ void __launch_bounds__(kCholThreads) k_chol_coop(Fit f) {
    __shared__ int s_i[kCholRows], s_off[kCholRows + 1];
    __shared__ double s_a[kCholRows];
    __shared__ int s_ok;
    const int p = f.p, tid = threadIdx.x, b = blockIdx.x, G = gridDim.x;
    double* U = f.cmat;
    int* ready = f.scratch;   // ready[k] = 1: row k final (zeroed by the host)
    for (int k = 0; k < p; ++k) {
        if (tid == 0) {
            int ok = 1;
            if (k > 0) {
                ok = wait_flag_set(ready + k, f.ctl) ? 1 : 0;
                __threadfence();
            }
            s_ok = ok;
        }
        __syncthreads();   // also orders this CTA's writes of step k - 1 before its reads
        if (!s_ok) return;
        const double* uk = U + size_t(k) * p;
        const double ukk = __ldcg(uk + k);
        if (!(ukk > 0.0)) {
            if (tid == 0 && b == k % G) set_status(f.ctl, LINGAM_EDEGENERATE);
            return;
        }
        const double inv = 1.0 / ukk;
        // row k + 1 first, published as soon as it is final
        const int i1 = k + 1;
        if (i1 < p && i1 % G == b) {
            chol_rows(U, uk, inv, p, i1, p, s_i, s_off, s_a);   // stride p: this row alone
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                atomicExch(ready + i1, 1);
            }
        }
        if (b == k % G) {
            const double rk = sqrt(ukk);
            for (int i = k + tid; i < p; i += kCholThreads) f.rmat[size_t(k) * p + i] = __ldcg(uk + i) / rk;
        }
        // this CTA's other rows i > k + 1 (i = b mod G), in blocks of kCholRows
        const int ifirst = k + 2 + ((b - (k + 2)) % G + G) % G;
        for (int i0 = ifirst; i0 < p; i0 += kCholRows * G) chol_rows(U, uk, inv, p, i0, G, s_i, s_off, s_a);
    }
}

// Column j of R^{-1} by forward substitution (one CTA per column):
//   y_k = ([k == j] - sum_{m<k} R[k][m] y_m) / R[k][k],  k = j..p-1.
// For p <= NT kTriPer, thread t owns the entries i = t, t + NT, ... of the running sums, in
// registers; column k + 1 of R is loaded while step k runs, so a step's critical path is one
// barrier, a shared-memory read and a few FMAs; and the diagonal's reciprocals are formed
// first, all at once (FP64 divisions are slow on this part).  Larger p: the plain loop.
constexpr int kTriThreads = 256;
constexpr int kTriPer = 4;
__global__ void __launch_bounds__(kTriThreads) k_tri_inv(Fit f) {
    extern __shared__ double sm_tri[];
    double* acc = sm_tri;        // [p] running sums (entries of other threads read at step k)
    const int p = f.p, j = blockIdx.x, tid = threadIdx.x;
    for (int i = tid; i < p; i += kTriThreads) acc[i] = 0.0;
    if (p <= kTriThreads * kTriPer) {
        double* invd = sm_tri + p;   // [p] 1 / R[k][k]
        for (int i = tid; i < p; i += kTriThreads) invd[i] = i >= j ? 1.0 / f.rmat[size_t(i) * p + i] : 0.0;
        __syncthreads();
        double a[kTriPer], cur[kTriPer];
#pragma unroll
        for (int q = 0; q < kTriPer; ++q) {
            a[q] = 0.0;
            const int i = tid + q * kTriThreads;
            cur[q] = i < p ? f.rmat[size_t(j) * p + i] : 0.0;
        }
        for (int k = j; k < p; ++k) {
            double nxt[kTriPer];
            if (k + 1 < p) {
#pragma unroll
                for (int q = 0; q < kTriPer; ++q) {
                    const int i = tid + q * kTriThreads;
                    nxt[q] = i < p ? __ldg(f.rmat + size_t(k + 1) * p + i) : 0.0;
                }
            }
            const double y = ((k == j ? 1.0 : 0.0) - acc[k]) * invd[k];
            if (tid == 0) f.rinv[size_t(k) * p + j] = y;
#pragma unroll
            for (int q = 0; q < kTriPer; ++q) {
                const int i = tid + q * kTriThreads;
                if (i > k && i < p) {
                    a[q] = fma(cur[q], y, a[q]);
                    if (i == k + 1) acc[i] = a[q];   // the only sum step k + 1 reads
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < kTriPer; ++q) cur[q] = nxt[q];
        }
    } else {
        __syncthreads();
        for (int k = j; k < p; ++k) {
            const double* rk = f.rmat + size_t(k) * p;   // column k of R: rk[i] = R[i][k]
            const double y = ((k == j ? 1.0 : 0.0) - acc[k]) / rk[k];
            if (tid == 0) f.rinv[size_t(k) * p + j] = y;
            for (int i = k + 1 + tid; i < p; i += kTriThreads) acc[i] = fma(rk[i], y, acc[i]);
            __syncthreads();
        }
    }
}

// B[K[a]][K[b]] = -R[a][a] Rinv[a][b] for a > b, 0 elsewhere.
__global__ void k_B_out(Fit f) {
    const int p = f.p;
    const int a = blockIdx.y * 16 + (threadIdx.x >> 4), b = blockIdx.x * 16 + (threadIdx.x & 15);
    if (a >= p || b >= p) return;
    const double v = a > b ? -f.rmat[size_t(a) * p + a] * f.rinv[size_t(a) * p + b] : 0.0;
    f.bout[size_t(f.order[a]) * p + f.order[b]] = v;
}

// The same fit for a problem of p <= kBSmall in one CTA (batches: one CTA per
// problem): C in shared memory, Cholesky C = L L^T in place (L lower, L = R), then
// thread b solves column b of L^{-1} by forward substitution into the problem's rinv
// (column-major, scratch) and writes B[K[a]][K[b]] = -L[a][a] Linv[a][b] for a > b.
// Problems with p > kBSmall, or whose status is bad, are left to other launches.
constexpr int kBSmall = 128;
constexpr int kBThreads = 256;

__global__ void __launch_bounds__(kBThreads) k_bfit_small(const Fit* __restrict__ fits, int count) {
    extern __shared__ double C[];
    const Fit f = fits[blockIdx.x];
    const int p = f.p, tid = threadIdx.x;
    if (p > kBSmall || ((volatile Ctl*)f.ctl)->status != 0) return;
    for (int idx = tid; idx < p * p; idx += kBThreads) {
        const int a = idx / p, b = idx - a * p;
        const int ia = f.order[a], ib = f.order[b];
        C[idx] = f.sd[ia] * f.sd[ib] * f.sig0[size_t(ia) * p + ib];
    }
    __syncthreads();
    for (int k = 0; k < p; ++k) {
        const double ckk = C[k * p + k];
        if (!(ckk > 0.0)) {   // every thread reads the same value: a uniform exit
            if (tid == 0) set_status(f.ctl, LINGAM_EDEGENERATE);
            return;
        }
        const double rk = sqrt(ckk);
        __syncthreads();
        for (int i = k + 1 + tid; i < p; i += kBThreads) C[i * p + k] /= rk;
        if (tid == 0) C[k * p + k] = rk;
        __syncthreads();
        const int m = p - k - 1;
        for (int idx = tid; idx < m * m; idx += kBThreads) {
            const int i = k + 1 + idx / m, j = k + 1 + idx % m;
            if (j <= i) C[i * p + j] -= C[i * p + k] * C[j * p + k];
        }
        __syncthreads();
    }
    double* y = f.rinv;   // column b of L^{-1} at y[b * p + a], a >= b
    for (int b = tid; b < p; b += kBThreads) {
        const int kb = f.order[b];
        for (int a = 0; a < b; ++a) f.bout[size_t(f.order[a]) * p + kb] = 0.0;
        for (int a = b; a < p; ++a) {
            double acc = a == b ? 1.0 : 0.0;
            for (int m2 = b; m2 < a; ++m2) acc = fma(-C[a * p + m2], y[size_t(b) * p + m2], acc);
            const double ya = acc / C[a * p + a];
            y[size_t(b) * p + a] = ya;
            f.bout[size_t(f.order[a]) * p + kb] = a > b ? -C[a * p + a] * ya : 0.0;
        }
    }
}

cudaError_t launch_fit_B_batch(const Fit* fits_dev, const int* p_host, int count, const Fit* fits_host,
                               cudaStream_t st) {
    int pmax_small = 0;
    for (int k = 0; k < count; ++k)
        if (p_host[k] <= kBSmall && p_host[k] > pmax_small) pmax_small = p_host[k];
    if (pmax_small > 0) {
        const size_t smem = size_t(pmax_small) * pmax_small * sizeof(double);
        cudaError_t e = ensure_smem_attr(reinterpret_cast<const void*>(k_bfit_small), smem);
        if (e != cudaSuccess) return e;
        k_bfit_small<<<count, kBThreads, smem, st>>>(fits_dev, count);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    for (int k = 0; k < count; ++k)
        if (p_host[k] > kBSmall) {
            const cudaError_t e = launch_fit_B(fits_host[k], st);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

cudaError_t launch_fit_B(const Fit& f, cudaStream_t st) {
    const int p = f.p;
    dim3 g2((p + 15) / 16, (p + 15) / 16);
    k_perm_cov<<<g2, 256, 0, st>>>(f);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_chol_coop, kCholThreads, 0)) != cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if ((e = cudaMemsetAsync(f.scratch, 0, size_t(p) * sizeof(int), st)) != cudaSuccess) return e;   // row flags
    {
        // one CTA per SM at most (co-resident: cooperative launch), no more than rows
        const int grid = std::max(1, std::min(nsm, p));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(kCholThreads);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if ((e = cudaLaunchKernelEx(&cfg, k_chol_coop, f)) != cudaSuccess) return e;
    }
    const size_t smem = (p <= kTriThreads * kTriPer ? 2 : 1) * size_t(p) * sizeof(double);
    e = ensure_smem_attr(reinterpret_cast<const void*>(k_tri_inv), smem);
    if (e != cudaSuccess) return e;
    k_tri_inv<<<p, kTriThreads, smem, st>>>(f);
    k_B_out<<<g2, 256, 0, st>>>(f);
    return cudaGetLastError();
}

}  // namespace lingam

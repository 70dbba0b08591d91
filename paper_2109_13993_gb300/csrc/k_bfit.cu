// k_bfit.cu -- causal strengths B from the causal order (Algorithm 1, last
// line; "conventional covariance-based regression", Sec. II-C), FP64.
//
// B row K[k] holds the least-squares coefficients of x_{K[k]} on its
// predecessors x_{K[0..k-1]}.  With C the covariance of the original variables
// permuted into the order K and C = R R^T its Cholesky factorisation (R lower
// triangular), the innovations e = diag(R) R^{-1} x are uncorrelated and
// x = (I - diag(R) R^{-1}) x + e, so B_K = I - diag(R) R^{-1}, strictly lower
// triangular; B is B_K with rows and columns mapped back to variable indices.
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

// Right-looking Cholesky, step k: column k of R (stored as row k of Rt = rmat)
// and the Schur-complement update of the trailing lower triangle.
__global__ void k_chol_step(Fit f, int k) {
    const int p = f.p;
    const double ckk = f.cmat[size_t(k) * p + k];
    if (!(ckk > 0.0)) {
        if (threadIdx.x == 0 && blockIdx.x == 0 && blockIdx.y == 0) set_status(f.ctl, LINGAM_EDEGENERATE);
        return;
    }
    if (blockIdx.x == 0 && blockIdx.y == 0) {
        const double rk = sqrt(ckk);
        for (int i = k + threadIdx.x; i < p; i += blockDim.x) f.rmat[size_t(k) * p + i] = f.cmat[size_t(i) * p + k] / rk;
    }
    const int i = k + 1 + blockIdx.y * 16 + (threadIdx.x >> 4);
    const int j = k + 1 + blockIdx.x * 16 + (threadIdx.x & 15);
    if (i >= p || j > i) return;
    f.cmat[size_t(i) * p + j] -= f.cmat[size_t(i) * p + k] * f.cmat[size_t(j) * p + k] / ckk;
}

// Column j of R^{-1} by forward substitution (one CTA per column):
//   y_k = ([k == j] - sum_{m<k} R[k][m] y_m) / R[k][k],  k = j..p-1.
__global__ void k_tri_inv(Fit f) {
    extern __shared__ double acc[];
    const int p = f.p, j = blockIdx.x, tid = threadIdx.x;
    for (int i = tid; i < p; i += blockDim.x) acc[i] = 0.0;
    __syncthreads();
    for (int k = j; k < p; ++k) {
        const double* rk = f.rmat + size_t(k) * p;   // column k of R: rk[i] = R[i][k]
        const double y = ((k == j ? 1.0 : 0.0) - acc[k]) / rk[k];
        if (tid == 0) f.rinv[size_t(k) * p + j] = y;
        for (int i = k + 1 + tid; i < p; i += blockDim.x) acc[i] = fma(rk[i], y, acc[i]);
        __syncthreads();
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

cudaError_t launch_fit_B(const Fit& f, cudaStream_t st) {
    const int p = f.p;
    dim3 g2((p + 15) / 16, (p + 15) / 16);
    k_perm_cov<<<g2, 256, 0, st>>>(f);
    for (int k = 0; k < p; ++k) {
        const int m = p - k - 1;
        dim3 g(m > 0 ? (m + 15) / 16 : 1, m > 0 ? (m + 15) / 16 : 1);
        k_chol_step<<<g, 256, 0, st>>>(f, k);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = size_t(p) * sizeof(double);
    e = ensure_smem_attr(reinterpret_cast<const void*>(k_tri_inv), smem);
    if (e != cudaSuccess) return e;
    k_tri_inv<<<p, 256, smem, st>>>(f);
    k_B_out<<<g2, 256, 0, st>>>(f);
    return cudaGetLastError();
}

}  // namespace lingam

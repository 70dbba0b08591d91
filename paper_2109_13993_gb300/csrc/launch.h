// launch.h -- host-side launchers of the CUDA kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace lingam {

// Raises the dynamic shared-memory limit of `func` to `bytes` once per device.
cudaError_t ensure_smem_attr(const void* func, size_t bytes);


// Normalise the rows of the input (Alg. 3 line 3), write the padded working copy,
// the row moments and H(x) - H(nu).
cudaError_t launch_standardize(const Fit& f, const void* x, int input_dtype, cudaStream_t st);
// Sigma = Xn Xn^T / (n-1) of the normalised rows (Alg. 3 line 4); sig0 = sig.
cudaError_t launch_gram(const Fit& f, cudaStream_t st);
// Start of iteration `it`: candidate order, score reset, first wave.
cudaError_t launch_plan(const Fit& f, int it, int nsplit, cudaStream_t st);
// One wave of pair comparisons (and, in its last CTA, the wave finalisation).
cudaError_t launch_pair_wave(const Fit& f, int it, int grid, cudaStream_t st);
// Remove the root from the data (Alg. 7) and from the covariance (Alg. 8).
cudaError_t launch_remove_root(const Fit& f, int it, int r, cudaStream_t st);
// B from the order: Cholesky of the covariance in causal order, B = I - diag(R) R^{-1}.
cudaError_t launch_fit_B(const Fit& f, cudaStream_t st);

}  // namespace lingam

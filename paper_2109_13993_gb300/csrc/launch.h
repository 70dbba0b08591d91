// launch.h -- host-side launchers of the CUDA kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace lingam {

// Raises the dynamic shared-memory limit of `func` to `bytes` once per device.
cudaError_t ensure_smem_attr(const void* func, size_t bytes);


// Normalise the rows of the input (NormalizeData, Algorithm 3), write the padded working copy,
// the row moments and H(x) - H(nu).
cudaError_t launch_standardize(const Fit& f, const void* x, int input_dtype, cudaStream_t st);
// Batch start: per-problem init (orders unset, counters zero) and NormalizeData of all
// rows of `count` problems (rowoff[d] = first global row of problem d, `rows` in all).
cudaError_t launch_standardize_batch(const Fit* fits, const SrcDesc* src, const int* rowoff, int count, int rows,
                                     int precision, int input_dtype, cudaStream_t st);
// Sigma = Xn Xn^T / (n-1) of the normalised rows (CalculateCovMat, Algorithm 3); sig0 = sig.
cudaError_t launch_gram(const Fit& f, cudaStream_t st);
// The same product on the tensor cores (mixed path): the rows are split into exact
// TF32 digits (three p x ld float planes and p exponents in `digits`), tcgen05 MMAs
// over 128 x 128 tiles of the upper triangle with the sample axis split over CTAs,
// float-float partial tiles in `partial`, summed in FP64 into sig and sig0.
cudaError_t launch_gram_tc(const Fit& f, void* digits, void* partial, cudaStream_t st);
// The mixed path's Gram of every problem with p <= kSmallGramP and row length ld <=
// kSmallGramLd of a batch table of up to kBatchLaunchMax problems, in one launch of `units`
// CTAs (gram_small_batch_units of the table's p and ld); exact FP32 products summed in
// float-float.  The other problems are skipped.
constexpr int kSmallGramP = 128;
constexpr int kSmallGramLd = 2048;
int gram_small_batch_units(const long long* p, const int* ld, int count);
cudaError_t launch_gram_small_batch(const Fit* fits_dev, int count, int units, cudaStream_t st);
// Bytes of `digits` and of `partial` that launch_gram_tc needs for p variables and row length ld.
size_t gram_tc_digit_bytes(long long p, int ld);
size_t gram_tc_partial_bytes(long long p, int ld);
// One iteration of Algorithm 3 (ParaFindRoot, UpdateData, UpdateCovMat) as one
// persistent cooperative launch; grid = SMs.
cudaError_t launch_iteration(const Fit& f, int it, int grid, cudaStream_t st);
// Largest co-resident grid of the iteration kernel (one CTA per SM).
int iteration_grid(const Fit& f, int nsm);
// The ordering of up to 512 problems (a Fit table in device memory, each with its own
// control block) in one persistent cooperative launch, all iterations, in lockstep;
// bctl carries the launch's barrier, abort flag and timeout.  The mixed path's pair tiles
// are tile_rows x tile_cols (64 x 32, 32 x 32 or 64 x 16; every Fit of the table carries
// the same shape); the FP64 path's are 32 x 32.
cudaError_t launch_batch(const Fit* fits_dev, int count, int maxp, int precision, int tile_rows, int tile_cols,
                         Ctl* bctl, int nsm, cudaStream_t st);
constexpr int kBatchLaunchMax = 512;   // problems per launch_batch
// B from the order: Cholesky of the covariance in causal order, B = I - diag(R) R^{-1}.
cudaError_t launch_fit_B(const Fit& f, cudaStream_t st);
// Bounded-wait self-test (k_iter.cu): the status the wait recorded (LINGAM_ETIMEOUT expected).
cudaError_t run_wait_selftest(int which, unsigned long long timeout_ns, int* status, cudaStream_t st);
// B of many problems: one CTA per problem of p <= 128 (shared-memory Cholesky), the
// multi-launch fit for larger ones.  p_host and fits_host mirror the device table.
cudaError_t launch_fit_B_batch(const Fit* fits_dev, const int* p_host, int count, const Fit* fits_host,
                               cudaStream_t st);

// Pair-tile autotuner (autotune.cu): the tile shape of the mixed path for a problem
// size, recording a measured choice, and forgetting all of them.
struct TileShape {
    int rows, cols;
};
TileShape autotune_tile_shape(long long p, long long n);
void autotune_record(long long p, long long n, TileShape shape);
void autotune_clear();
// The same for batch calls, keyed by the batch's largest p and largest n.
TileShape autotune_batch_shape(long long maxp, long long maxn);
void autotune_batch_record(long long maxp, long long maxn, TileShape shape);

}  // namespace lingam

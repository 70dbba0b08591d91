/*
 * lingam.h -- C ABI of the GB300 DirectLiNGAM causal-ordering library.
 *
 * Problem statement (ParaLiNGAM paper, Sec. II-B and II-C): the input is a
 * data matrix X of p variables by n samples, row i holding the n samples of
 * variable X_i; the model is X = B X + N with B strictly lower triangular in
 * some causal order (Eq. base_mat).  The library returns a causal order K
 * (Algorithm 1) and the weighted adjacency matrix B estimated from K by
 * ordinary least squares of every variable on its predecessors.
 *
 * Each iteration (Algorithm 3) compares every still-unordered pair of
 * normalised variables with the likelihood-ratio measure of Eq. Itest, using
 * the entropy approximation of Eq. HApp and the closed-form normalised
 * residual of Eq. var_update, adds min(0, I)^2 to the scores (Algorithm 2),
 * takes the variable of lowest score as the root, and removes it from the
 * data (Algorithm 7, UpdateData) and from the covariance matrix (Eq.
 * CovUpdate, Algorithm 8).  A pair is evaluated once for both directions
 * (messaging, Sec. III-A: I(j,i) = -I(i,j)) and a variable stops being
 * compared once its partial score exceeds the best complete score (threshold,
 * Sec. III-B); both shortcuts leave the result unchanged.
 *
 * Conventions for every entry point:
 *   - Errors are returned as lingam_status codes; nothing is thrown across
 *     the ABI.  Outputs are written only when the call returns LINGAM_OK.
 *   - The caller owns every buffer, the workspace included.  The library
 *     allocates no device memory for data.  State kept between calls: the
 *     pair-tile autotuner's table (lingam_autotune), the address of the
 *     static scratch area (lingam_fit_static), the executable graphs of batch
 *     calls (lingam_fit_batch, lingam_fit_bootstrap; keyed by workspace and
 *     shapes; at most 32 are kept, and capturing one more destroys the least
 *     recently launched idle one) and, per host thread and device, the CUDA
 *     events of the calls (created once, reused by every call) and eight
 *     streams and their events for the independent per-problem launches of a
 *     batch.
 *   - Data pointers may point to host or device memory; the library tells
 *     them apart with cudaPointerGetAttributes.  Host buffers are copied
 *     inside the call.  All device work is ordered on opts->stream (a batch
 *     forks the covariances of its problems above 128 variables or 2048
 *     samples onto the library's streams and joins them back into it; the
 *     smaller problems' covariances are one launch on opts->stream) and the
 *     call returns after that stream has drained (it is synchronous).
 *   - The device is the CUDA device current on the calling thread.
 *   - Environment variables, read by the library: LINGAM_LOG=1 prints one
 *     line per call on stderr (entry point, sizes, status); LINGAM_FAULT=<step>
 *     makes the named step of every call report a failed launch (host-side
 *     fault injection for testing: standardize, covariance, iteration:<k>,
 *     bfit, batch); LINGAM_NARROW=<rows> sets the fewest rows for which a wave
 *     of 16 columns or fewer of a 64 x 32 single fit runs on 128 x 16 tiles
 *     (default 256; 0 turns these narrow waves off, a switch for measurement).
 */
#ifndef LINGAM_H
#define LINGAM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LINGAM_OK = 0,
    LINGAM_EINVAL = -1,       /* bad argument: p < 1, n < 3, NULL pointer, bad option, workspace too small */
    LINGAM_EDEGENERATE = -2,  /* zero variance row or residual, non-finite data, or a pair with
                                 1 - rho^2 <= 2^-20 (mixed path) / 1e-14 (FP64 path): collinear */
    LINGAM_ENOMEM = -3,       /* reserved: the library itself never allocates */
    LINGAM_ECUDA = -4,        /* a CUDA runtime call or kernel launch failed */
    LINGAM_ETIMEOUT = -5,     /* a bounded device-side wait ran out (opts.timeout_s) */
    LINGAM_EBOUNDS = -6       /* debug build only (LINGAM_BOUNDS_CHECK): an index bound check of a
                                 kernel failed; the access was skipped */
} lingam_status;

/* opts.precision */
enum { LINGAM_FP64 = 0, LINGAM_MIXED = 1 };
/* opts.input_dtype */
enum { LINGAM_F32 = 0, LINGAM_F64 = 1 };

typedef struct {
    int precision;           /* LINGAM_MIXED (FP32 pair measure, FP64 covariance and B) or LINGAM_FP64 */
    int input_dtype;         /* element type of X: LINGAM_F32 or LINGAM_F64 */
    int prune;               /* 1 = threshold pruning (Sec. III-B), 0 = compare every pair */
    int reuse;               /* 1 = one evaluation per unordered pair (Sec. III-A), 0 = every ordered pair */
    int tile_i, tile_j;      /* pair-tile shape of the mixed path, rows x columns: 64 x 32, 32 x 32 or
                                64 x 16, and for batch calls only 32 x 16 and 1 x 1 (one pair per warp)
                                (a zero in one takes 64 rows or 32 columns); both 0 = the autotuner's
                                table (lingam_tile_rows/_cols, lingam_batch_tile_rows/_cols).  The FP64
                                path uses 32 x 32. */
    int split_n;             /* single fits: split of the sample axis.  0 (default) = stream-K over
                                (tile, 32-sample group) units: a wave's units are spread over the whole
                                grid, so a tile's samples are cut into as many CTA segments as it takes
                                to fill every SM.  s > 0 = at most ntiles * s CTAs work on a wave, so a
                                tile is cut into about s segments (s = 1: one CTA per tile while a wave
                                has fewer tiles than SMs).  Results move by FP32 rounding only (the
                                partial moments of a tile are summed over its segments in fixed order).
                                Ignored by the batch entry points. */
    double timeout_s;        /* bound on any device-side wait; <= 0 means 10 s */
    void* stream;            /* cudaStream_t to run on; NULL = the legacy default stream */
    const int* forced_order; /* NULL, or p variable indices (host memory): iteration k takes
                                forced_order[k] as its root instead of the argmin; scores are still
                                those of the current iteration.  Used for iteration-by-iteration checks. */
    int max_iters;           /* 0 = all p iterations; else stop after this many (order[k] = -1 beyond,
                                B is then not computed).  Used to time a bounded prefix of a run. */
    int timing;              /* 1 = also time every iteration's launch (report t_pair_ms and
                                t_pair_iter_ms; one CUDA event recorded after each launch) and
                                run the device phase timers (t_compute_ms ...); 0 for production */
    const signed char* prior; /* NULL, or a p x p HOST matrix of prior knowledge (the paper notes
                                that DirectLiNGAM accepts prior knowledge, Sec. II-C; read as known
                                ancestors): prior[i*p + j] = 1 says X_j is known to be an ancestor
                                of X_i; 0 or -1 say nothing to the ordering.  At every iteration
                                only variables with no known ancestor left unordered may be the
                                root; every remaining variable is still compared with them, and
                                the scores of the others are reported as NaN.  Values other than
                                -1, 0, 1, or a cycle among the known ancestors: LINGAM_EINVAL.
                                Single fits only (lingam_fit, lingam_fit_static, lingam_autotune). */
    double gamma0;           /* 0 (default): threshold pruning against the lowest complete score of the
                                iteration so far (exact, Sec. III-B).  > 0: the paper's own schedule
                                instead (Sec. III-B, III-C; Algorithm 6 and the host loop of
                                Algorithm 9), for ablation: each iteration starts with threshold
                                gamma = gamma0; a variable whose partial score exceeds gamma stops
                                taking new partners; when no variable is left to go on and none
                                finished at or below gamma, gamma is multiplied by gamma_c until some
                                variable can go on (or one that finished lies below it), and the
                                stopped variables at or below the new gamma go on.  The root is
                                the same as with gamma0 = 0 (both thresholds are exact); pairs
                                evaluated and report.threshold_updates show the schedule's cost.
                                Needs prune = reuse = 1; single fits only; NaN, negative or
                                infinite: LINGAM_EINVAL. */
    double gamma_c;          /* growth factor of gamma (> 1; default 2), used when gamma0 > 0 */
} lingam_opts;

typedef struct {
    /* Each of these is NULL or a HOST array the library fills in. */
    double* root_score;          /* [p] score S of the root chosen at iteration k */
    double* margin_lb;           /* [p] lower bound of (second lowest score - root score) at iteration k;
                                    +inf when a single variable is left */
    long long* pairs_evaluated;  /* [p] pair evaluations at iteration k (unordered pairs when reuse = 1) */
    double* scores;              /* [p*p] scores[k*p + v]: S_v at iteration k if v was compared with every
                                    other remaining variable at that iteration; NaN if v was already
                                    ordered or was pruned before completing */
    /* Filled in whenever the report pointer is non-NULL (device time, CUDA events). */
    double t_standardize_ms, t_gram_ms, t_order_ms, t_B_ms;
    long long pairs_total;       /* sum of pairs_evaluated over the run */
    long long pairs_unpruned;    /* sum over iterations of r(r-1)/2 (r(r-1) when reuse = 0) */
    double t_pair_ms;            /* device time of the pair-comparison launches (opts.timing = 1), else 0 */
    long long kernel_launches;   /* kernels this call launched */
    double* t_pair_iter_ms;      /* NULL or a HOST array [p]: with opts.timing = 1, the time of the
                                    launch of iteration k, between the stream events recorded after
                                    launch k - 1 (before the first launch) and after launch k */
    /* With opts.timing = 1 (single fits): device wall time (CTA 0's global timer, summed
       over all iterations) of CTA 0's own pair-compute phases of the waves, of the rest of
       each wave as CTA 0 sees it (the wait for the slower CTAs' tiles, the merge and the
       finalisation, up to the wave's published result), and of CTA 0's part of the
       removals (UpdateData, UpdateCovMat).  0 otherwise. */
    double t_compute_ms, t_merge_ms, t_remove_ms;
    long long threshold_updates; /* opts.gamma0 > 0: times the threshold was multiplied by gamma_c,
                                    summed over the iterations (each one a kernel launch and a
                                    read-back in the paper's host loop, Algorithm 9); else 0 */
    long long waves;             /* pair waves run over the fit (single fits) */
    long long tile_pairs;        /* pairs the waves' tiles computed: tiles x rows x columns, row
                                    padding, unused columns and the duplicate half of the
                                    columns' own block included (pairs_total are the useful ones) */
    long long empty_col_pairs;   /* of tile_pairs: those in column slots a wave left empty */
    long long pad_row_pairs;     /* of tile_pairs: those of the padding rows of a wave's last tile */
} lingam_report;

/* Fills *opts with the defaults: MIXED, F32, prune = reuse = 1, autotuned
 * tiles, timeout 10 s, default stream, no forced order, all iterations, no
 * per-iteration timing. */
void lingam_default_opts(lingam_opts* opts);

/* Size in bytes of the device workspace lingam_fit needs for a p x n problem
 * with these options (NULL = defaults).  Returns 0 for invalid sizes.  The
 * workspace must be device memory aligned to 256 bytes. */
size_t lingam_workspace_size(long long p, long long n, const lingam_opts* opts);

/*
 * lingam_fit -- DirectLiNGAM (Algorithm 1) accelerated as in Algorithm 3.
 *   X          p x n row-major samples, element type opts->input_dtype; host or device.
 *   p, n       p >= 1 variables, n >= 3 samples.
 *   order      [p] ints, host or device: order[k] = 0-based index of the k-th variable of the
 *              causal order; order[0] is the first root (most exogenous variable).
 *   B          [p*p] doubles, host or device, or NULL: B[i*p + j] = b_ij, the direct effect of X_j
 *              on X_i in the units of X (Eq. base_linear); strictly lower triangular once rows
 *              and columns are permuted into `order`.
 *   workspace  device memory of at least lingam_workspace_size(p, n, opts) bytes.
 *   opts       NULL = defaults.
 *   report     NULL or a report to fill in.
 * Returns LINGAM_OK or an error status.
 */
int lingam_fit(const void* X, long long p, long long n, int* order, double* B, void* workspace,
               const lingam_opts* opts, lingam_report* report);

/*
 * lingam_covariance -- NormalizeData and CalculateCovMat of Algorithm 3 alone: the
 * covariance matrix of the normalised rows, Sigma = Xn Xn^T / (n-1), where row i of Xn
 * is (X_i - mean) / sd with the divisor n-1 in the variance (Eq. var_update).
 *   X, p, n, workspace, opts  as in lingam_fit (opts->forced_order must be NULL).
 *   Sigma      [p*p] doubles, host or device, row-major; Sigma[i*p + i] = 1 exactly.
 *   report     NULL, or a report whose t_standardize_ms, t_gram_ms and kernel_launches
 *              are filled in (the other fields are left untouched).
 * precision LINGAM_MIXED computes the product on the tensor cores from a TF32 + FP32
 * split of the FP32 rows (FP32 accumulation, FP64 sum of the sample-axis splits);
 * LINGAM_FP64 computes it in FP64.  Sigma is written only on LINGAM_OK; rows with zero
 * variance or non-finite values give LINGAM_EDEGENERATE.
 */
int lingam_covariance(const void* X, long long p, long long n, double* Sigma, void* workspace,
                      const lingam_opts* opts, lingam_report* report);

/*
 * Pair-tile autotuner (the paper has no counterpart: its GPU design has one tile shape).
 * The mixed path evaluates pairs in tiles of rows x columns variables: 64 x 32 (512
 * threads), 32 x 32 or 64 x 16 (256 threads, two CTAs per SM).  The columns of a tile are
 * the candidates a wave completes, so 16-column tiles prune more finely (fewer pairs, more
 * waves).  Which shape is faster depends on p, n and the data.  The library keeps a
 * process-wide table of the choice per size bucket (ceil(log2 p), ceil(log2 n)); a
 * bucket never measured uses 64 x 32.
 *
 * lingam_tile_rows, lingam_tile_cols -- the shape lingam_fit uses for a p x n problem
 *                       when opts->tile_i and opts->tile_j are 0.
 * lingam_autotune    -- measures the ordering of X (as lingam_fit with opts, B not
 *                       fitted) once with each shape, records the fastest for X's size
 *                       bucket and returns it in *tile_rows, *tile_cols; ms[0..2] (if
 *                       ms is not NULL) receive the ordering times with 64 x 32, 32 x 32
 *                       and 64 x 16 tiles.  Costs three fits; the workspace is as for
 *                       lingam_fit.
 * lingam_batch_tile_rows, lingam_batch_tile_cols -- the shape lingam_fit_batch and
 *                       lingam_fit_bootstrap use on the mixed path for a batch whose
 *                       largest problem has maxp variables and maxn samples, when
 *                       opts->tile_i and opts->tile_j are 0.  Batches have a table of their
 *                       own (bucket of the largest p and n); a bucket never measured uses
 *                       the pair mode, 1 x 1, when maxp <= 128 (it was the fastest shape on
 *                       every measured batch of small problems), else 32 x 32.  With
 *                       opts->reuse = 0 the pair mode runs as 64 x 16.
 * lingam_autotune_batch -- measures lingam_fit_batch on the caller's count datasets (as
 *                       lingam_fit_batch with opts on the mixed path, B not fitted) with
 *                       each shape: a warm-up call, the call that captures the graph, and
 *                       the timed third call (host wall time of the synchronous call).
 *                       Batches have two more shapes for many small problems: 32 x 16
 *                       tiles (128 threads, three CTAs per SM, 64-sample chunks), and the
 *                       pair mode, 1 x 1, in which every pair a wave needs is evaluated
 *                       whole by one warp (no tile, so no pair slot is computed in vain;
 *                       waves of up to 16 columns).  Records the fastest for the bucket of
 *                       the batch's largest p and n, returns it in *tile_rows, *tile_cols,
 *                       and ms[0..4] (if not NULL) receive the times with 64 x 32, 32 x 32,
 *                       64 x 16, 32 x 16 and 1 x 1.  Costs fifteen batch calls; the
 *                       workspace is as for lingam_fit_batch.  LINGAM_EINVAL for the FP64
 *                       path.
 * lingam_autotune_reset -- forgets every measured choice (both tables).
 * The tables are shared by all threads of the process (guarded by a mutex).
 */
int lingam_tile_rows(long long p, long long n);
int lingam_tile_cols(long long p, long long n);
int lingam_autotune(const void* X, long long p, long long n, void* workspace, const lingam_opts* opts,
                    int* tile_rows, int* tile_cols, double* ms);
int lingam_batch_tile_rows(long long maxp, long long maxn);
int lingam_batch_tile_cols(long long maxp, long long maxn);
int lingam_autotune_batch(int count, const void* const* X, const long long* p, const long long* n, void* workspace,
                          const lingam_opts* opts, int* tile_rows, int* tile_cols, double* ms);
void lingam_autotune_reset(void);

/*
 * lingam_selftest_wait -- failure detection check: one of the library's device-side waits,
 * made to wait for an event that never happens, must give up after timeout_s seconds and
 * record LINGAM_ETIMEOUT in its control block, and the kernel must end normally (the context
 * stays usable).  which = 0: an mbarrier phase that no thread completes (the copy-ring waits
 * of the iteration and batch kernels); 1: the grid barrier with its arrival count started one
 * arrival off, two CTAs (the barrier of the iteration and batch kernels); 2: the wave word of
 * a single fit that nothing publishes; 3: a row flag of the B fit's Cholesky that nothing
 * sets.  The control block and flag are library-owned device variables.  *observed receives
 * the recorded status.  Returns LINGAM_EINVAL for which outside 0..3, timeout_s outside
 * (0, 60] or a NULL observed, LINGAM_ECUDA if the launch fails, else LINGAM_OK.  Synchronous
 * on the legacy default stream.
 */
int lingam_selftest_wait(int which, double timeout_s, int* observed);

/* Workspace for lingam_fit_batch over `count` datasets of sizes p[k] x n[k]. */
size_t lingam_workspace_size_batch(int count, const long long* p, const long long* n, const lingam_opts* opts);

/*
 * lingam_fit_batch -- `count` independent problems of uneven p and n (Algorithm 3 on
 * each; the paper fits one dataset at a time).  X[k], p[k], n[k], order[k], B[k] as in
 * lingam_fit for dataset k; B may be NULL (no B for any dataset) and a B[k] may be
 * NULL (no B for that one).  status[k] (host array, may be NULL) receives each
 * dataset's status; report may be NULL or an array of `count` reports (their time
 * fields are set to -1: the datasets run together).  Returns the first non-OK dataset
 * status, else LINGAM_OK.  A dataset that turns out degenerate does not stop the
 * others; a timeout stops all of them.
 *
 * All problems run in one persistent cooperative launch per 512 problems, in
 * lockstep over iterations: each wave's pair tiles of all problems are partitioned
 * over the whole GPU together.  The device work of a call is captured into a CUDA
 * graph on the second call with the same workspace and problem shapes (and options),
 * and replayed by every later such call; calls on the legacy default stream (NULL)
 * run without a graph.  opts->forced_order and opts->prior must be NULL, and
 * opts->max_iters and opts->gamma0 0; opts->split_n is ignored.  Pair tiles: on the
 * mixed path opts->tile_i x opts->tile_j for every problem of the call (64 x 32, 32 x 32,
 * 64 x 16, 32 x 16, or 1 x 1: one pair per warp, which needs opts->reuse = 1 and otherwise
 * runs 64 x 16), or, with both 0, the batch autotuner's shape for the largest p and n
 * (lingam_batch_tile_rows/_cols); 32 x 32 on the FP64 path.
 */
int lingam_fit_batch(int count, const void* const* X, const long long* p, const long long* n, int* const* order,
                     double* const* B, void* workspace, const lingam_opts* opts, int* status,
                     lingam_report* report);

/* Workspace for lingam_fit_bootstrap of nboot resamples of a p x n dataset. */
size_t lingam_workspace_size_bootstrap(long long p, long long n, int nboot, const lingam_opts* opts);

/*
 * lingam_fit_bootstrap -- nboot bootstrap resamples of one dataset, as lingam_fit_batch.
 *   X       p x n row-major samples (opts->input_dtype), host or device, read in place
 *           (copied once if on the host).
 *   idx     nboot x n int indices in [0, n), host or device: resample b is the p x n
 *           matrix whose column t is column idx[b n + t] of X (observations drawn with
 *           replacement); the library draws no random numbers.
 *   order   nboot x p ints, host or device: order[b p + k] as lingam_fit's order[k].
 *   B       NULL or nboot x p x p doubles: resample b's B at B + b p p.
 *   status, report as lingam_fit_batch (arrays of nboot).
 * The gather of the resampled columns is fused into the normalisation of the rows.
 */
int lingam_fit_bootstrap(const void* X, long long p, long long n, int nboot, const int* idx, int* order, double* B,
                         void* workspace, const lingam_opts* opts, int* status, lingam_report* report);

/*
 * lingam_fit_static -- lingam_fit for callers that cannot allocate device memory.
 *
 * The paper has no counterpart to this entry point; it exists for callers
 * that have no way to provide the device workspace lingam_fit needs: a plain
 * host program without a device allocator of its own, a plug-in inside an
 * application whose memory pool owns the GPU, or a code path where calling
 * the CUDA allocator is not allowed.  It computes exactly what lingam_fit
 * computes, with the same arguments minus the workspace, in a scratch array
 * of LINGAM_STATIC_SCRATCH_BYTES that the library holds on every GPU it is
 * loaded on until the process exits.  It allocates nothing.
 *
 *   - Returns LINGAM_EINVAL when lingam_workspace_size(p, n, opts) exceeds
 *     LINGAM_STATIC_SCRATCH_BYTES (32 MiB).  With the default options (and FP64
 *     input for the FP64 path) that admits: the mixed path up to p = 128 at
 *     n = 10^4, p = 217 at n = 5000, p = 430 at n = 1000; the FP64 path up to
 *     p = 74 at n = 10^4, p = 136 at n = 5000, p = 333 at n = 1000.  The
 *     workspace grows about linearly in n (the rows) and in p^2 (the
 *     covariances), so lingam_workspace_size is the test for other sizes.
 *   - The first call on a device looks up the scratch array's device address
 *     (once per device, with that device current); make that first call before
 *     any stream capture on the device.
 *   - Every call on a device uses the same scratch array and leaves its
 *     contents behind; each call initialises what it needs.  Calls whose GPU
 *     work overlaps (several host threads, or several streams) race on the
 *     array: serialise them.
 */
#define LINGAM_STATIC_SCRATCH_BYTES (32u << 20)
int lingam_fit_static(const void* X, long long p, long long n, int* order, double* B, const lingam_opts* opts,
                      lingam_report* report);

/* Static, human-readable name of a status code. */
const char* lingam_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* LINGAM_H */

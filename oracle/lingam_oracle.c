/*
 * lingam_oracle.c -- plain, slow FP64 CPU DirectLiNGAM.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, constant table or helper with the CUDA path.
 *
 * What it computes (ParaLiNGAM paper, Sec. II-C):
 *   Algorithm 1 (DirectLiNGAM): K = [], U = all variables; repeat
 *     root = FindRoot(X, U); append root to K; remove it from U;
 *     X = RegressRoot(X, U, root)
 *   until U is empty (the printed "until U is not empty" is read as "until U
 *   is empty": p iterations, the last one trivial); then B from K.
 *   Algorithm 2 (FindRoot): for every ordered pair (i, j), i != j in U:
 *     normalise x_i and x_j, regress each on the other, normalise both
 *     residuals, S[i] += min(0, I(x_i, x_j, r_i^(j), r_j^(i)))^2;
 *     root = U[argmin S] (lowest variable index on ties).
 *   Eq. Itest: I = H(x_j) + H(r_i^(j)) - H(x_i) - H(r_j^(i)).
 *   Eq. HApp:  H(u) = H(nu) - k1 [E log cosh u - beta]^2 - k2 [E u exp(-u^2/2)]^2,
 *              H(nu) = (1 + log 2 pi) / 2, k1 = 79.047, k2 = 7.4129,
 *              beta = 0.37457 (the printed values, used as is).
 *   Sec. III-E residual definition: r_i^(j) = x_i - cov(x_i,x_j)/var(x_j) x_j.
 *
 * Readings where the paper is silent:
 *   - "Normalize" = subtract the sample mean, divide by the sample standard
 *     deviation with divisor n-1 (the divisor of Eq. var_update); E{.} in
 *     Eq. HApp is the plain sample mean (divisor n).
 *   - cov and var use divisor n-1 and explicit two-pass centring.
 *   - The normalised x_i is the same for every partner j, so it and H(x_i)
 *     are computed once per FindRoot call instead of once per pair; every
 *     residual is still regressed and normalised explicitly per ordered pair.
 *   - RegressRoot regresses each remaining x_w on x_root by explicit OLS on
 *     the samples of the current (unnormalised) data.
 *   - B: "conventional covariance-based regression" is read as ordinary
 *     least squares of each variable on all of its predecessors in K, on
 *     the original centred data, solved from the normal equations by
 *     Gaussian elimination with partial pivoting.
 *   - Degenerate input (a zero-variance row or residual, a non-finite value)
 *     makes the call fail with ORACLE_EDEGENERATE.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_EDEGENERATE (-2)
#define ORACLE_ENOMEM (-3)

static const double ORACLE_K1 = 79.047;
static const double ORACLE_K2 = 7.4129;
static const double ORACLE_BETA = 0.37457;

double oracle_const_k1(void) { return ORACLE_K1; }
double oracle_const_k2(void) { return ORACLE_K2; }
double oracle_const_beta(void) { return ORACLE_BETA; }
double oracle_const_h_gauss(void) { return 0.5 * (1.0 + log(2.0 * M_PI)); }

/* Sample mean (divisor n). */
static double mean_of(const double* x, long n) {
    double s = 0.0;
    for (long t = 0; t < n; ++t) s += x[t];
    return s / (double)n;
}

/* Sample covariance, divisor n-1, explicit centring. */
static double cov_of(const double* x, const double* y, long n) {
    double mx = mean_of(x, n), my = mean_of(y, n), s = 0.0;
    for (long t = 0; t < n; ++t) s += (x[t] - mx) * (y[t] - my);
    return s / (double)(n - 1);
}

/* Normalize: out = (x - mean) / sd, sd with divisor n-1.  Returns 0 or
 * ORACLE_EDEGENERATE for zero variance / non-finite data. */
int oracle_standardize(const double* x, long n, double* out) {
    double m = mean_of(x, n), v = 0.0;
    for (long t = 0; t < n; ++t) v += (x[t] - m) * (x[t] - m);
    v /= (double)(n - 1);
    if (!(v > 0.0) || !isfinite(v)) return ORACLE_EDEGENERATE;
    double sd = sqrt(v);
    for (long t = 0; t < n; ++t) out[t] = (x[t] - m) / sd;
    return ORACLE_OK;
}

/* CalculateCovMat (Algorithm 3) by its definition: every row normalised as
 * above, then Sigma[i][j] = sum_t xn_i[t] xn_j[t] / (n-1), both triangles
 * computed (the diagonal too, so it is 1 only up to rounding).  X is p x n
 * row-major, out p x p row-major. */
int oracle_covariance(const double* X, int p, long n, double* out) {
    double* Z = (double*)malloc(sizeof(double) * (size_t)p * (size_t)n);
    if (!Z) return ORACLE_ENOMEM;
    for (int i = 0; i < p; ++i) {
        int st = oracle_standardize(X + (size_t)i * n, n, Z + (size_t)i * n);
        if (st != ORACLE_OK) {
            free(Z);
            return st;
        }
    }
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j) {
            const double* zi = Z + (size_t)i * n;
            const double* zj = Z + (size_t)j * n;
            double s = 0.0;
            for (long t = 0; t < n; ++t) s += zi[t] * zj[t];
            out[(size_t)i * p + j] = s / (double)(n - 1);
        }
    free(Z);
    return ORACLE_OK;
}

/* Eq. HApp on an already normalised sample u. */
double oracle_entropy(const double* u, long n) {
    double lc = 0.0, g = 0.0;
    for (long t = 0; t < n; ++t) {
        lc += log(cosh(u[t]));
        g += u[t] * exp(-u[t] * u[t] / 2.0);
    }
    lc /= (double)n;
    g /= (double)n;
    double a = lc - ORACLE_BETA;
    return oracle_const_h_gauss() - ORACLE_K1 * a * a - ORACLE_K2 * g * g;
}

/* Residual of x regressed on y by OLS: r = x - cov(x,y)/var(y) y. */
int oracle_regress(const double* x, const double* y, long n, double* r) {
    double vy = cov_of(y, y, n);
    if (!(vy > 0.0)) return ORACLE_EDEGENERATE;
    double b = cov_of(x, y, n) / vy;
    for (long t = 0; t < n; ++t) r[t] = x[t] - b * y[t];
    return ORACLE_OK;
}

/* Compare (Alg. 2, the body of the pair loop) on already normalised xi, xj
 * with their entropies hi = H(xi), hj = H(xj).  work holds 2n doubles. */
static int compare_normalised(const double* xi, const double* xj, double hi, double hj, long n,
                              double* work, double* I_out) {
    double* ri = work;
    double* rj = work + n;
    int st;
    if ((st = oracle_regress(xi, xj, n, ri)) != ORACLE_OK) return st;
    if ((st = oracle_regress(xj, xi, n, rj)) != ORACLE_OK) return st;
    if ((st = oracle_standardize(ri, n, ri)) != ORACLE_OK) return st;
    if ((st = oracle_standardize(rj, n, rj)) != ORACLE_OK) return st;
    double I = hj + oracle_entropy(ri, n) - hi - oracle_entropy(rj, n);
    if (!isfinite(I)) return ORACLE_EDEGENERATE;
    *I_out = I;
    return ORACLE_OK;
}

/* I(x_i, x_j, r_i^(j), r_j^(i)) of Eq. Itest for two raw sample rows. */
int oracle_pair_measure(const double* xi_raw, const double* xj_raw, long n, double* I_out) {
    if (n < 3) return ORACLE_EINVAL;
    double* w = (double*)malloc(sizeof(double) * 4 * (size_t)n);
    if (!w) return ORACLE_ENOMEM;
    int st = oracle_standardize(xi_raw, n, w);
    if (st == ORACLE_OK) st = oracle_standardize(xj_raw, n, w + n);
    if (st == ORACLE_OK)
        st = compare_normalised(w, w + n, oracle_entropy(w, n), oracle_entropy(w + n, n), n, w + 2 * n, I_out);
    free(w);
    return st;
}

/* ---------------- FindRoot over all ordered pairs, threaded over i -------------- */

typedef struct {
    const double* Z;     /* normalised rows, p x n */
    const double* H;     /* H(z_v) per variable */
    const int* U;        /* remaining variables */
    int r;
    long n;
    double* S;           /* scores, indexed by position in U */
    int next;            /* work counter (guarded by mu) */
    int status;
    pthread_mutex_t mu;
} findroot_job;

static void* findroot_worker(void* arg) {
    findroot_job* job = (findroot_job*)arg;
    long n = job->n;
    double* work = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    if (!work) {
        pthread_mutex_lock(&job->mu);
        job->status = ORACLE_ENOMEM;
        pthread_mutex_unlock(&job->mu);
        return NULL;
    }
    for (;;) {
        pthread_mutex_lock(&job->mu);
        int a = job->next++;
        int bad = job->status != ORACLE_OK;
        pthread_mutex_unlock(&job->mu);
        if (a >= job->r || bad) break;
        int i = job->U[a];
        double s = 0.0;
        for (int b = 0; b < job->r; ++b) {
            if (b == a) continue;
            int j = job->U[b];
            double I;
            int st = compare_normalised(job->Z + (size_t)i * n, job->Z + (size_t)j * n, job->H[i], job->H[j], n,
                                        work, &I);
            if (st != ORACLE_OK) {
                pthread_mutex_lock(&job->mu);
                job->status = st;
                pthread_mutex_unlock(&job->mu);
                break;
            }
            double m = I < 0.0 ? I : 0.0;
            s += m * m;
        }
        job->S[a] = s;
    }
    free(work);
    return NULL;
}

static int resolve_threads(int nthreads) {
    if (nthreads > 0) return nthreads;
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    return c > 0 ? (int)c : 1;
}

/* Scores of every variable in U (Alg. 2), S indexed by position in U. */
static int find_root_scores(const double* X, const int* U, int r, long n, int p, int nthreads, double* S) {
    double* Z = (double*)malloc(sizeof(double) * (size_t)p * (size_t)n);
    double* H = (double*)malloc(sizeof(double) * (size_t)p);
    if (!Z || !H) { free(Z); free(H); return ORACLE_ENOMEM; }
    int st = ORACLE_OK;
    for (int a = 0; a < r && st == ORACLE_OK; ++a) {
        int v = U[a];
        st = oracle_standardize(X + (size_t)v * n, n, Z + (size_t)v * n);
        if (st == ORACLE_OK) H[v] = oracle_entropy(Z + (size_t)v * n, n);
    }
    if (st == ORACLE_OK) {
        findroot_job job;
        job.Z = Z; job.H = H; job.U = U; job.r = r; job.n = n; job.S = S; job.next = 0; job.status = ORACLE_OK;
        pthread_mutex_init(&job.mu, NULL);
        int nt = resolve_threads(nthreads);
        if (nt > r) nt = r;
        pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nt);
        int started = 0;
        for (int k = 0; k < nt; ++k)
            if (pthread_create(&th[k], NULL, findroot_worker, &job) == 0) ++started;
        if (started == 0) findroot_worker(&job);
        for (int k = 0; k < started; ++k) pthread_join(th[k], NULL);
        free(th);
        pthread_mutex_destroy(&job.mu);
        st = job.status;
    }
    free(Z);
    free(H);
    return st;
}

/* Scores of every variable of U for one FindRoot call on raw rows X (p x n).
 * S_out is indexed by position in U. */
int oracle_find_root_scores(const double* X, int p, long n, const int* U, int r, int nthreads, double* S_out) {
    if (p < 1 || n < 3 || r < 1) return ORACLE_EINVAL;
    if (r == 1) { S_out[0] = 0.0; return ORACLE_OK; }
    return find_root_scores(X, U, r, n, p, nthreads, S_out);
}

/* ---------------- B: OLS of each variable on its predecessors in K ---------------- */

/* Solve A x = b (m x m, row-major) by Gaussian elimination with partial pivoting. */
static int gauss_solve(double* A, double* b, int m) {
    for (int c = 0; c < m; ++c) {
        int piv = c;
        for (int r = c + 1; r < m; ++r)
            if (fabs(A[(size_t)r * m + c]) > fabs(A[(size_t)piv * m + c])) piv = r;
        if (!(fabs(A[(size_t)piv * m + c]) > 0.0)) return ORACLE_EDEGENERATE;
        if (piv != c) {
            for (int k = 0; k < m; ++k) {
                double t = A[(size_t)c * m + k];
                A[(size_t)c * m + k] = A[(size_t)piv * m + k];
                A[(size_t)piv * m + k] = t;
            }
            double t = b[c]; b[c] = b[piv]; b[piv] = t;
        }
        for (int r = c + 1; r < m; ++r) {
            double f = A[(size_t)r * m + c] / A[(size_t)c * m + c];
            if (f == 0.0) continue;
            for (int k = c; k < m; ++k) A[(size_t)r * m + k] -= f * A[(size_t)c * m + k];
            b[r] -= f * b[c];
        }
    }
    for (int c = m - 1; c >= 0; --c) {
        double s = b[c];
        for (int k = c + 1; k < m; ++k) s -= A[(size_t)c * m + k] * b[k];
        b[c] = s / A[(size_t)c * m + c];
    }
    return ORACLE_OK;
}

/* B[i*p + j] = effect of X_j on X_i; row K[k] holds the OLS coefficients of
 * x_{K[k]} on x_{K[0..k-1]} (original data, covariances with divisor n-1). */
int oracle_fit_B(const double* X, int p, long n, const int* K, double* B) {
    if (p < 1 || n < 3) return ORACLE_EINVAL;
    double* C = (double*)malloc(sizeof(double) * (size_t)p * p);
    double* A = (double*)malloc(sizeof(double) * (size_t)p * p);
    double* rhs = (double*)malloc(sizeof(double) * (size_t)p);
    if (!C || !A || !rhs) { free(C); free(A); free(rhs); return ORACLE_ENOMEM; }
    for (int a = 0; a < p; ++a)
        for (int b = a; b < p; ++b) {
            double c = cov_of(X + (size_t)a * n, X + (size_t)b * n, n);
            C[(size_t)a * p + b] = c;
            C[(size_t)b * p + a] = c;
        }
    memset(B, 0, sizeof(double) * (size_t)p * p);
    int st = ORACLE_OK;
    for (int k = 1; k < p && st == ORACLE_OK; ++k) {
        int tgt = K[k];
        for (int a = 0; a < k; ++a) {
            for (int b = 0; b < k; ++b) A[(size_t)a * k + b] = C[(size_t)K[a] * p + K[b]];
            rhs[a] = C[(size_t)K[a] * p + tgt];
        }
        st = gauss_solve(A, rhs, k);
        if (st == ORACLE_OK)
            for (int a = 0; a < k; ++a) B[(size_t)tgt * p + K[a]] = rhs[a];
    }
    free(C); free(A); free(rhs);
    return st;
}

/* ---------------- Algorithm 1 ---------------- */

/* Prior knowledge (the paper notes that DirectLiNGAM accepts prior knowledge, Sec. II-C; it
 * is read here as known ancestors): prior[i*p + j] == 1 says that x_j is an ancestor of x_i.
 * At every iteration only the variables of U with no known ancestor left in U can be the
 * root; every variable of U stays a partner in the comparisons (Algorithm 2 unchanged). */
static int is_candidate(const signed char* prior, int p, const int* U, int r, int a) {
    if (!prior) return 1;
    for (int b = 0; b < r; ++b)
        if (b != a && prior[(size_t)U[a] * p + U[b]] == 1) return 0;
    return 1;
}

/*
 * oracle_fit: DirectLiNGAM on X (p x n, row-major, not modified).
 *   order[p]       causal order K (0-based variable indices), order[0] first root.
 *   B[p*p]         (nullable) weights, see oracle_fit_B.
 *   scores[p*p]    (nullable) scores[it*p + v] = S_v at iteration it for v in U,
 *                  NaN for variables already removed.
 *   forced[p]      (nullable) if given, iteration it takes forced[it] as its root
 *                  (scores are still those of FindRoot on the current U).
 *   nthreads       threads for FindRoot (0 = all online cores).
 */
static int fit_impl(const double* X, int p, long n, int* order, double* B, double* scores, const int* forced,
                    const signed char* prior, int nthreads) {
    if (p < 1 || n < 3 || !X || !order) return ORACLE_EINVAL;
    double* W = (double*)malloc(sizeof(double) * (size_t)p * (size_t)n);
    int* U = (int*)malloc(sizeof(int) * (size_t)p);
    double* S = (double*)malloc(sizeof(double) * (size_t)p);
    double* tmp = (double*)malloc(sizeof(double) * (size_t)n);
    if (!W || !U || !S || !tmp) { free(W); free(U); free(S); free(tmp); return ORACLE_ENOMEM; }
    memcpy(W, X, sizeof(double) * (size_t)p * (size_t)n);
    for (size_t e = 0; e < (size_t)p * (size_t)n; ++e)
        if (!isfinite(W[e])) { free(W); free(U); free(S); free(tmp); return ORACLE_EDEGENERATE; }
    for (int v = 0; v < p; ++v) U[v] = v;
    int r = p, st = ORACLE_OK;
    for (int it = 0; it < p && st == ORACLE_OK; ++it) {
        /* FindRoot */
        if (r == 1) S[0] = 0.0;
        else st = find_root_scores(W, U, r, n, p, nthreads, S);
        if (st != ORACLE_OK) break;
        int best = -1;
        for (int a = 0; a < r; ++a) {
            if (!is_candidate(prior, p, U, r, a)) continue;
            if (best < 0) best = a;
            else if (S[a] < S[best] || (S[a] == S[best] && U[a] < U[best])) best = a;
        }
        if (best < 0) { st = ORACLE_EINVAL; break; }   /* a cycle among the known ancestors */
        if (scores) {
            for (int v = 0; v < p; ++v) scores[(size_t)it * p + v] = NAN;
            for (int a = 0; a < r; ++a)
                if (is_candidate(prior, p, U, r, a)) scores[(size_t)it * p + U[a]] = S[a];
        }
        if (forced) {
            best = -1;
            for (int a = 0; a < r; ++a)
                if (U[a] == forced[it]) best = a;
            if (best < 0) { st = ORACLE_EINVAL; break; }
        }
        int root = U[best];
        order[it] = root;
        /* remove root from U, keep ascending variable order */
        for (int a = best; a + 1 < r; ++a) U[a] = U[a + 1];
        --r;
        /* RegressRoot: x_w <- x_w - cov(x_w, x_root)/var(x_root) x_root for w in U */
        for (int a = 0; a < r && st == ORACLE_OK; ++a) {
            int w = U[a];
            st = oracle_regress(W + (size_t)w * n, W + (size_t)root * n, n, tmp);
            if (st == ORACLE_OK) memcpy(W + (size_t)w * n, tmp, sizeof(double) * (size_t)n);
        }
    }
    if (st == ORACLE_OK && B) st = oracle_fit_B(X, p, n, order, B);
    free(W); free(U); free(S); free(tmp);
    return st;
}

int oracle_fit(const double* X, int p, long n, int* order, double* B, double* scores, const int* forced,
               int nthreads) {
    return fit_impl(X, p, n, order, B, scores, forced, NULL, nthreads);
}

/* oracle_fit with prior knowledge prior[p*p] (see is_candidate); scores of the variables
 * that cannot be the root at an iteration are NaN. */
int oracle_fit_prior(const double* X, int p, long n, const signed char* prior, int* order, double* B,
                     double* scores, const int* forced, int nthreads) {
    if (!prior) return ORACLE_EINVAL;
    return fit_impl(X, p, n, order, B, scores, forced, prior, nthreads);
}

/* I for a list of (i, j) variable pairs of raw rows X (p x n), threaded. */
typedef struct {
    const double* X; long n; const int* pi; const int* pj; int m; double* I; int next; int status;
    pthread_mutex_t mu;
} pairs_job;

static void* pairs_worker(void* arg) {
    pairs_job* job = (pairs_job*)arg;
    for (;;) {
        pthread_mutex_lock(&job->mu);
        int k = job->next++;
        pthread_mutex_unlock(&job->mu);
        if (k >= job->m) break;
        int st = oracle_pair_measure(job->X + (size_t)job->pi[k] * job->n, job->X + (size_t)job->pj[k] * job->n,
                                     job->n, &job->I[k]);
        if (st != ORACLE_OK) {
            pthread_mutex_lock(&job->mu);
            job->status = st;
            pthread_mutex_unlock(&job->mu);
        }
    }
    return NULL;
}

int oracle_pair_measures(const double* X, long n, const int* pi, const int* pj, int m, int nthreads, double* I) {
    if (n < 3 || m < 0) return ORACLE_EINVAL;
    pairs_job job;
    job.X = X; job.n = n; job.pi = pi; job.pj = pj; job.m = m; job.I = I; job.next = 0; job.status = ORACLE_OK;
    pthread_mutex_init(&job.mu, NULL);
    int nt = resolve_threads(nthreads);
    if (nt > m) nt = m > 0 ? m : 1;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nt);
    int started = 0;
    for (int k = 0; k < nt; ++k)
        if (pthread_create(&th[k], NULL, pairs_worker, &job) == 0) ++started;
    if (started == 0) pairs_worker(&job);
    for (int k = 0; k < started; ++k) pthread_join(th[k], NULL);
    free(th);
    pthread_mutex_destroy(&job.mu);
    return job.status;
}

int oracle_num_threads(int nthreads) { return resolve_threads(nthreads); }

/* ---------------- scores of selected variables after a given prefix of roots ---------------- */

typedef struct {
    const double* Z; const double* H; const int* U; int r; long n; const int* vars; int m; double* S;
    int next; int status; pthread_mutex_t mu;
} varscore_job;

static void* varscore_worker(void* arg) {
    varscore_job* job = (varscore_job*)arg;
    long n = job->n;
    double* work = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    if (!work) {
        pthread_mutex_lock(&job->mu); job->status = ORACLE_ENOMEM; pthread_mutex_unlock(&job->mu);
        return NULL;
    }
    /* work items: (variable k, partner position b); each item adds one term,
       summed per variable afterwards in partner order */
    for (;;) {
        pthread_mutex_lock(&job->mu);
        int item = job->next++;
        int bad = job->status != ORACLE_OK;
        pthread_mutex_unlock(&job->mu);
        if (item >= job->m * job->r || bad) break;
        int k = item / job->r, b = item % job->r;
        int i = job->vars[k], j = job->U[b];
        double term = 0.0;
        if (i != j) {
            double I;
            int st = compare_normalised(job->Z + (size_t)i * n, job->Z + (size_t)j * n, job->H[i], job->H[j], n,
                                        work, &I);
            if (st != ORACLE_OK) {
                pthread_mutex_lock(&job->mu); job->status = st; pthread_mutex_unlock(&job->mu);
                break;
            }
            double mneg = I < 0.0 ? I : 0.0;
            term = mneg * mneg;
        }
        job->S[item] = term;
    }
    free(work);
    return NULL;
}

/*
 * oracle_variable_scores: replay the roots prefix[0..k-1] on X (RegressRoot
 * after each, Alg. 1), then return S_v (Alg. 2) for each v in vars[0..m-1]
 * against the remaining set U.  out[m].  Every v must still be in U.
 */
int oracle_variable_scores(const double* X, int p, long n, const int* prefix, int k, const int* vars, int m,
                           int nthreads, double* out) {
    if (p < 1 || n < 3 || k < 0 || k >= p || m < 0) return ORACLE_EINVAL;
    double* W = (double*)malloc(sizeof(double) * (size_t)p * (size_t)n);
    int* U = (int*)malloc(sizeof(int) * (size_t)p);
    char* in = (char*)calloc((size_t)p, 1);
    double* tmp = (double*)malloc(sizeof(double) * (size_t)n);
    double* Z = (double*)malloc(sizeof(double) * (size_t)p * (size_t)n);
    double* H = (double*)malloc(sizeof(double) * (size_t)p);
    double* terms = (double*)malloc(sizeof(double) * ((size_t)m * p + 1));
    int st = ORACLE_OK;
    if (!W || !U || !in || !tmp || !Z || !H || !terms) st = ORACLE_ENOMEM;
    if (st == ORACLE_OK) {
        memcpy(W, X, sizeof(double) * (size_t)p * (size_t)n);
        for (int v = 0; v < p; ++v) in[v] = 1;
        for (int it = 0; it < k && st == ORACLE_OK; ++it) {
            int root = prefix[it];
            if (root < 0 || root >= p || !in[root]) { st = ORACLE_EINVAL; break; }
            in[root] = 0;
            for (int w = 0; w < p && st == ORACLE_OK; ++w) {
                if (!in[w]) continue;
                st = oracle_regress(W + (size_t)w * n, W + (size_t)root * n, n, tmp);
                if (st == ORACLE_OK) memcpy(W + (size_t)w * n, tmp, sizeof(double) * (size_t)n);
            }
        }
    }
    int r = 0;
    if (st == ORACLE_OK) {
        for (int v = 0; v < p; ++v) if (in[v]) U[r++] = v;
        for (int a = 0; a < m; ++a) if (vars[a] < 0 || vars[a] >= p || !in[vars[a]]) st = ORACLE_EINVAL;
    }
    for (int a = 0; a < r && st == ORACLE_OK; ++a) {
        int v = U[a];
        st = oracle_standardize(W + (size_t)v * n, n, Z + (size_t)v * n);
        if (st == ORACLE_OK) H[v] = oracle_entropy(Z + (size_t)v * n, n);
    }
    if (st == ORACLE_OK && m > 0) {
        varscore_job job;
        job.Z = Z; job.H = H; job.U = U; job.r = r; job.n = n; job.vars = vars; job.m = m; job.S = terms;
        job.next = 0; job.status = ORACLE_OK;
        pthread_mutex_init(&job.mu, NULL);
        int nt = resolve_threads(nthreads);
        pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nt);
        int started = 0;
        for (int t = 0; t < nt; ++t)
            if (pthread_create(&th[t], NULL, varscore_worker, &job) == 0) ++started;
        if (started == 0) varscore_worker(&job);
        for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
        free(th);
        pthread_mutex_destroy(&job.mu);
        st = job.status;
        if (st == ORACLE_OK)
            for (int a = 0; a < m; ++a) {
                double s = 0.0;
                for (int b = 0; b < r; ++b) s += terms[(size_t)a * r + b];
                out[a] = s;
            }
    }
    free(W); free(U); free(in); free(tmp); free(Z); free(H); free(terms);
    return st;
}

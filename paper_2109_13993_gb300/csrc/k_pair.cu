// k_pair.cu -- the pair comparison of one iteration (ParaFindRoot, Algorithm 4),
// one "wave" per launch, and the wave finalisation (scores, threshold, next
// wave, root selection) run by the last CTA of the wave.
//
// A wave pairs a block of up to kTJ candidate variables (the columns) with
// every variable that has not been a column yet in this iteration (the rows;
// the columns themselves come first among the rows so that pairs inside the
// block are covered too).  Each unordered pair is evaluated once and its
// measure I(i,j) of Eq. Itest serves both variables (messaging, Sec. III-A:
// I(j,i) = -I(i,j)).  After the wave its columns have met every other
// variable, so their scores (Algorithm 2) are complete.  The lowest complete
// score bounds the root's score (threshold, Sec. III-B): a variable whose
// partial score exceeds it can no longer be the root and is never made a
// column, so pairs of two such variables are never evaluated.  The iteration
// ends when no live variable is left un-columned; the root is the complete
// variable of lowest score (lowest index on ties).
//
// Per pair and sample the kernel forms the two normalised residuals of Eq.
// var_update / Algorithm 7 from the covariance rho = Sigma[i,j]:
//   a = (x_i - rho x_j)/sqrt(1-rho^2) = r_i^(j),  b = (x_j - rho x_i)/sqrt(1-rho^2) = r_j^(i),
// and accumulates for each of them the two sample moments of Eq. HApp:
//   sum log cosh u  with  log cosh u = |u| + ln(1 + e^{-2|u|}) - ln 2,
//   sum u e^{-u^2/2}.
// The logarithm is taken once per group of kSub samples, of the product of the
// factors 1 + e^{-2|u|}, so in FP32 a sample costs two SFU base-2 exponentials
// per residual.  Group sums are centred (log cosh u - beta), which keeps the
// running FP32 sums small; the group and split structure is a cascaded
// (blocked pairwise) summation.
#include <type_traits>

#include "common.cuh"
#include "launch.h"
#include "tma.cuh"

namespace lingam {

template <class T>
struct PairCfg;
template <>
struct PairCfg<float> {
    static constexpr int CH = kChunk;
    static constexpr int LDS = kChunk + 4;    // padded smem row: conflict-free 16-byte loads
};
template <>
struct PairCfg<double> {
    static constexpr int CH = kChunk64;
    static constexpr int LDS = kChunk64 + 2;  // padded smem row
};

template <class T>
__host__ __device__ constexpr size_t stage_elems() {
    return size_t(kTI + kTJ) * PairCfg<T>::LDS;
}
template <class T>
size_t pair_smem_bytes() {
    return size_t(kStages) * stage_elems<T>() * sizeof(T) + kStages * sizeof(uint64_t);
}

// FP32 residuals carry the scale kScale: with u' = kScale*u,
//   e^{-u^2/2} = 2^{-u'^2},   e^{-2|u|} = 2^{kC3 |u'|}.
constexpr float kScale = 0.84932180028801904272f;     // sqrt(log2(e)/2)
constexpr float kInvScale = 1.17741002251547469101f;  // 1/kScale
constexpr float kC3 = -3.39728720115207617088f;       // -2 log2(e) / kScale

// ------------------------------------------------------------------ wave finalisation
__device__ void wave_finalize(const Fit& f, int it, int* red) {
    Ctl* ctl = f.ctl;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int ncol = ctl->ncol, nrow = ctl->nrow, ntiles = ctl->ntiles;
    const int p = f.p, r = ctl->r;

    // 1. row contributions: min(0, I(row, col))^2 summed over the wave's columns
    if (f.reuse)
        for (int e = tid; e < nrow; e += nth) f.part[f.rows[e]] += f.rowsum[e];
    __syncthreads();
    // 2. column contributions max(0, I(row, col))^2 = min(0, I(col, row))^2, tile order
    if (tid < ncol) {
        double tot = 0.0;
        for (int t = 0; t < ntiles; ++t) tot += f.colsum[t * kTJ + tid];
        const int v = f.cols[tid];
        f.part[v] += tot;
        f.flags[v] |= kColumned;
        if (f.want_scores) f.rep_scores[(size_t)it * p + v] = f.part[v];
    }
    __syncthreads();
    // 3. threshold = lowest complete score (lowest variable index on ties)
    if (tid == 0) {
        double best = ctl->best;
        int bv = ctl->best_var;
        for (int c = 0; c < ncol; ++c) {
            const int v = f.cols[c];
            const double s = f.part[v];
            if (bv < 0 || s < best || (s == best && v < bv)) {
                best = s;
                bv = v;
            }
        }
        ctl->best = best;
        ctl->best_var = bv;
        ctl->pairs_it += f.reuse ? (long long)ncol * (ncol - 1) / 2 + (long long)ncol * (nrow - ncol)
                                 : (long long)ncol * (nrow - 1);
    }
    __syncthreads();
    const double best = ctl->best;

    // 4. prune, then pick the next columns: the first kTJ live un-columned variables
    //    in candidate order.
    int nc = 0;
    for (int base = 0; base < r; base += nth) {
        const int k = base + tid;
        int live = 0, v = -1;
        if (k < r) {
            v = f.sigma[k];
            int fl = f.flags[v];
            if (!(fl & kColumned)) {
                if (!(fl & kDead) && f.prune && f.reuse && f.part[v] > best) {
                    fl |= kDead;
                    f.flags[v] = fl;
                }
                live = (fl & kDead) ? 0 : 1;
            }
        }
        int tot;
        const int rank = nc + block_scan01(live, red, &tot);
        if (live && rank < kTJ) {
            f.cols[rank] = v;
            f.flags[v] |= kPick;
        }
        nc += tot;
        __syncthreads();
    }
    nc = nc < kTJ ? nc : kTJ;
    __syncthreads();
    // 5. rows of the next wave: the columns, then every other row-eligible variable
    //    (un-columned ones with reuse; all remaining ones without) in candidate order.
    int nr = 0;
    for (int base = 0; base < r; base += nth) {
        const int k = base + tid;
        int take = 0, v = -1;
        if (k < r) {
            v = f.sigma[k];
            const int fl = f.flags[v];
            take = !(fl & kPick) && (!f.reuse || !(fl & kColumned));
        }
        int tot;
        const int rank = nr + block_scan01(take, red, &tot);
        if (take) f.scratch[rank] = v;
        nr += tot;
        __syncthreads();
    }
    __syncthreads();
    for (int k = tid; k < nc + nr; k += nth) {
        const int v = k < nc ? f.cols[k] : f.scratch[k - nc];
        f.rows[k] = v;
    }
    for (int c = tid; c < nc; c += nth) f.flags[f.cols[c]] &= ~kPick;
    __syncthreads();

    if (tid == 0) {
        if (nc == 0) {
            // 6. root = complete variable of lowest score (or the forced one)
            int root = f.has_forced ? f.forced[it] : ctl->best_var;
            double second = INFINITY;
            for (int k = 0; k < r; ++k) {
                const int v = f.sigma[k];
                if (v == ctl->best_var) continue;
                const double s = f.part[v];   // full score if complete, else a lower bound
                if (s < second) second = s;
            }
            ctl->root = root;
            ctl->done = 1;
            f.order[it] = root;
            f.rep_root_score[it] = f.part[root];
            f.rep_margin[it] = second - ctl->best;
            f.rep_pairs[it] = ctl->pairs_it;
        } else {
            ctl->ncol = nc;
            ctl->nrow = nc + nr;
            ctl->ntiles = (nc + nr + kTI - 1) / kTI;
            ctl->wave += 1;
        }
        ctl->wave_ctas_done = 0;
    }
}

// ------------------------------------------------------------------ the pair-wave kernel
template <class T>
__global__ void __launch_bounds__(kPairThreads, (sizeof(T) == 4 ? 2 : 1)) k_pair_wave(Fit f, int it) {
    using Cfg = PairCfg<T>;
    constexpr int CH = Cfg::CH, LDS = Cfg::LDS;
    constexpr bool kF32 = std::is_same<T, float>::value;
    Ctl* ctl = f.ctl;
    if (ctl->done || ctl->status != 0) return;
    const int S = ctl->nsplit;
    const int tile = blockIdx.x / S, split = blockIdx.x % S;
    const int ntiles = ctl->ntiles;
    if (tile >= ntiles) return;
    const int ncol = ctl->ncol, nrow = ctl->nrow;
    const int tid = threadIdx.x;
    const int ty = tid >> 4, tx = tid & 15;
    const int p = f.p, ld = f.ld;
    const T* __restrict__ xt = static_cast<const T*>(f.xt);

    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* stage_base = reinterpret_cast<T*>(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + size_t(kStages) * stage_elems<T>() * sizeof(T));
    __shared__ int s_rowvar[kTI], s_colvar[kTJ];
    __shared__ int s_flag;
    __shared__ int s_red[kPairThreads / 32];

    if (tid < kTI) {
        const int e = tile * kTI + tid;
        s_rowvar[tid] = e < nrow ? f.rows[e] : -1;
    } else if (tid < kTI + kTJ) {
        const int c = tid - kTI;
        s_colvar[c] = c < ncol ? f.cols[c] : -1;
    }
    // samples of this split: chunks [ch0, ch0 + nch)
    const int nch_total = ld / CH;
    const int nch_per = (nch_total + S - 1) / S;
    const int ch0 = split * nch_per;
    const int nch = max(0, min(nch_total, ch0 + nch_per) - ch0);

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
        fence_barrier_init();
    }
    __syncthreads();
    // empty slots are never copied into: zero them once
    for (int s = 0; s < kStages; ++s) {
        T* st = stage_base + size_t(s) * stage_elems<T>();
        for (int k = tid; k < (kTI + kTJ) * LDS; k += kPairThreads) {
            const int slot = k / LDS;
            const bool empty = slot < kTI ? (s_rowvar[slot] < 0) : (s_colvar[slot - kTI] < 0);
            if (empty) st[k] = T(0);
        }
    }
    __syncthreads();

    int issued = 0;   // chunks whose copies have been issued (thread 0 only)
    auto issue = [&](int chunk) {
        const int s = chunk % kStages;
        T* st = stage_base + size_t(s) * stage_elems<T>();
        const size_t t0 = size_t(ch0 + chunk) * CH;
        uint32_t bytes = 0;
        for (int e = 0; e < kTI; ++e) bytes += s_rowvar[e] >= 0 ? CH * sizeof(T) : 0;
        for (int c = 0; c < kTJ; ++c) bytes += s_colvar[c] >= 0 ? CH * sizeof(T) : 0;
        fence_proxy_async();
        mbar_expect_tx(&bars[s], bytes);
        for (int e = 0; e < kTI; ++e) {
            const int v = s_rowvar[e];
            if (v >= 0) bulk_g2s(st + e * LDS, xt + size_t(v) * ld + t0, CH * sizeof(T), &bars[s]);
        }
        for (int c = 0; c < kTJ; ++c) {
            const int v = s_colvar[c];
            if (v >= 0) bulk_g2s(st + (kTI + c) * LDS, xt + size_t(v) * ld + t0, CH * sizeof(T), &bars[s]);
        }
        issued = chunk + 1;
    };
    if (tid == 0)
        for (int c = 0; c < min(nch, kStages); ++c) issue(c);

    // per-pair constants; pair q = (row slot ty + 16*(q>>1), column slot tx + 16*(q&1))
    const int rsl[2] = {ty, ty + 16}, csl[2] = {tx, tx + 16};
    bool valid[4];
    T s_[4], sr_[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int e_loc = rsl[q >> 1], c = csl[q & 1];
        const int e = tile * kTI + e_loc;
        const int vi = s_rowvar[e_loc], vj = s_colvar[c];
        bool ok = vi >= 0 && vj >= 0;
        if (ok) ok = f.reuse ? (e >= ncol || c < e) : (vi != vj);
        valid[q] = ok;
        double rho = ok ? f.sig[size_t(vi) * p + vj] : 0.0;
        double om = fma(-rho, rho, 1.0);   // 1 - rho^2 in FP64
        if (ok && !(om > 1e-14)) {
            set_status(ctl, LINGAM_EDEGENERATE);
            om = 1.0;
            rho = 0.0;
        }
        if constexpr (kF32) {
            const float sc = kScale / sqrtf(float(om));
            s_[q] = sc;
            sr_[q] = sc * float(rho);
        } else {
            const double sc = 1.0 / sqrt(om);
            s_[q] = sc;
            sr_[q] = sc * rho;
        }
    }

    // accumulators, index 2q + 0 for a = r_i^(j) and 2q + 1 for b = r_j^(i):
    // A = sum |u|, P = prod (1 + e^{-2|u|}), G = sum u e^{-u^2/2} over the current group;
    // D = sum over closed groups of (log cosh u - beta), Gt = sum of closed-group G.
    T A[8], P[8], G[8], D[8], Gt[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        A[k] = T(0);
        P[k] = T(1);
        G[k] = T(0);
        D[k] = T(0);
        Gt[k] = T(0);
    }
    const T grp_off = T(-double(kSub) * (kLn2 + kBeta));

    bool ok_pipe = true;
    int c = 0;
    for (; c < nch; ++c) {
        const int s = c % kStages;
        ok_pipe = mbar_wait_bounded(&bars[s], (c / kStages) & 1, ctl, ctl->timeout_ns);
        if (__syncthreads_or(!ok_pipe)) {
            ok_pipe = false;
            break;
        }
        const T* st = stage_base + size_t(s) * stage_elems<T>();
        const T* R0 = st + rsl[0] * LDS;
        const T* R1 = st + rsl[1] * LDS;
        const T* C0 = st + (kTI + csl[0]) * LDS;
        const T* C1 = st + (kTI + csl[1]) * LDS;
        if constexpr (kF32) {
#pragma unroll 1
            for (int t = 0; t < CH; t += kSub) {
#pragma unroll 2
                for (int u = 0; u < kSub; u += 4) {
                    const float4 xr0 = *reinterpret_cast<const float4*>(R0 + t + u);
                    const float4 xr1 = *reinterpret_cast<const float4*>(R1 + t + u);
                    const float4 xc0 = *reinterpret_cast<const float4*>(C0 + t + u);
                    const float4 xc1 = *reinterpret_cast<const float4*>(C1 + t + u);
                    const float xi[2][4] = {{xr0.x, xr0.y, xr0.z, xr0.w}, {xr1.x, xr1.y, xr1.z, xr1.w}};
                    const float xj[2][4] = {{xc0.x, xc0.y, xc0.z, xc0.w}, {xc1.x, xc1.y, xc1.z, xc1.w}};
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float a = fmaf(s_[q], xi[q >> 1][k], -sr_[q] * xj[q & 1][k]);
                            const float b = fmaf(s_[q], xj[q & 1][k], -sr_[q] * xi[q >> 1][k]);
                            const float ga = ex2_approx(-a * a);
                            const float gb = ex2_approx(-b * b);
                            G[2 * q] = fmaf(a, ga, G[2 * q]);
                            G[2 * q + 1] = fmaf(b, gb, G[2 * q + 1]);
                            const float aa = fabsf(a), bb = fabsf(b);
                            const float ea = ex2_approx(aa * kC3);
                            const float eb = ex2_approx(bb * kC3);
                            P[2 * q] = fmaf(P[2 * q], ea, P[2 * q]);
                            P[2 * q + 1] = fmaf(P[2 * q + 1], eb, P[2 * q + 1]);
                            A[2 * q] += aa;
                            A[2 * q + 1] += bb;
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {   // close the group of kSub samples
                    D[k] += fmaf(float(kLn2), lg2_approx(P[k]), fmaf(A[k], kInvScale, grp_off));
                    Gt[k] += G[k];
                    A[k] = 0.f;
                    P[k] = 1.f;
                    G[k] = 0.f;
                }
            }
        } else {
#pragma unroll 1
            for (int t = 0; t < CH; t += kSub) {
#pragma unroll 1
                for (int u = 0; u < kSub; ++u) {
                    const double xi[2] = {R0[t + u], R1[t + u]};
                    const double xj[2] = {C0[t + u], C1[t + u]};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const double a = fma(s_[q], xi[q >> 1], -sr_[q] * xj[q & 1]);
                        const double b = fma(s_[q], xj[q & 1], -sr_[q] * xi[q >> 1]);
                        const double aa = fabs(a), bb = fabs(b);
                        P[2 * q] = fma(P[2 * q], exp(-2.0 * aa), P[2 * q]);
                        P[2 * q + 1] = fma(P[2 * q + 1], exp(-2.0 * bb), P[2 * q + 1]);
                        A[2 * q] += aa;
                        A[2 * q + 1] += bb;
                        G[2 * q] = fma(a, exp(-0.5 * a * a), G[2 * q]);
                        G[2 * q + 1] = fma(b, exp(-0.5 * b * b), G[2 * q + 1]);
                    }
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    D[k] += A[k] + log(P[k]) + grp_off;
                    Gt[k] += G[k];
                    A[k] = 0.0;
                    P[k] = 1.0;
                    G[k] = 0.0;
                }
            }
        }
        __syncthreads();   // every thread is done with stage s
        if (tid == 0 && c + kStages < nch) issue(c + kStages);
    }
    if (!ok_pipe) {
        // A wait ran out (status already recorded).  Give the copies still in flight a
        // bounded chance to land before the CTA releases its shared memory.
        if (tid == 0)
            for (int c2 = c; c2 < issued; ++c2) {
                const unsigned long long t0 = global_ns();
                while (!mbar_try_wait(&bars[c2 % kStages], (c2 / kStages) & 1) && global_ns() - t0 < 2000000000ull) {
                }
            }
        __syncthreads();
        return;
    }

    // ---- this split's partial moments
    T* parts = static_cast<T*>(f.partials);
    {
        T* dst = parts + ((size_t(tile) * S + split) * kPairThreads + tid) * 16;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            dst[4 * q + 0] = D[2 * q];
            dst[4 * q + 1] = Gt[2 * q];
            dst[4 * q + 2] = D[2 * q + 1];
            dst[4 * q + 3] = Gt[2 * q + 1];
        }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) s_flag = (atomicAdd(&f.tile_cnt[tile], 1) == S - 1);
    __syncthreads();
    if (!s_flag) return;
    __threadfence();

    // ---- last split of the tile: merge the splits in split order, evaluate I
    //      (Eq. Itest with Eq. HApp), reduce rows and columns in a fixed order.
    const double n = double(f.n);
    const double pad_fix = double(ld - f.n) * kBeta;   // each zero padding sample added -beta to D
    T* Ism = reinterpret_cast<T*>(smem_raw);           // [kTI][kTJ+1]; the stages are free now
    {
        T tot[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) tot[k] = T(0);
        for (int s2 = 0; s2 < S; ++s2) {
            const T* src = parts + ((size_t(tile) * S + s2) * kPairThreads + tid) * 16;
#pragma unroll
            for (int k = 0; k < 16; ++k) tot[k] += __ldcg(src + k);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e_loc = rsl[q >> 1], cc = csl[q & 1];
            T I = T(0);
            if (valid[q]) {
                const int vi = s_rowvar[e_loc], vj = s_colvar[cc];
                if constexpr (kF32) {
                    const float inv_n = float(1.0 / n);
                    const float ha = hterm_f(tot[4 * q + 0] + float(pad_fix), tot[4 * q + 1] * kInvScale, inv_n);
                    const float hb = hterm_f(tot[4 * q + 2] + float(pad_fix), tot[4 * q + 3] * kInvScale, inv_n);
                    I = (float(f.hx[vj]) - float(f.hx[vi])) + (ha - hb);
                } else {
                    const double ha = hterm(tot[4 * q + 0] + pad_fix, tot[4 * q + 1], n);
                    const double hb = hterm(tot[4 * q + 2] + pad_fix, tot[4 * q + 3], n);
                    I = (f.hx[vj] - f.hx[vi]) + (ha - hb);
                }
                if (!isfinite(double(I))) set_status(ctl, LINGAM_EDEGENERATE);
            }
            Ism[e_loc * (kTJ + 1) + cc] = I;
        }
    }
    __syncthreads();
    // Contributions are squared and summed in FP64 so that a variable's score
    // does not depend on how its pairs were grouped into tiles and waves.
    if (tid < kTI) {
        const int e = tile * kTI + tid;
        double s = 0.0;
        for (int cc = 0; cc < kTJ; ++cc) {
            const double I = double(Ism[tid * (kTJ + 1) + cc]);
            const double m = I < 0.0 ? I : 0.0;
            s = fma(m, m, s);
        }
        if (e < nrow) f.rowsum[e] = s;
    } else if (tid < kTI + kTJ) {
        const int cc = tid - kTI;
        double s = 0.0;
        for (int e = 0; e < kTI; ++e) {
            const double I = double(Ism[e * (kTJ + 1) + cc]);
            const double m = I > 0.0 ? I : 0.0;
            s = fma(m, m, s);
        }
        f.colsum[tile * kTJ + cc] = s;
    }
    if (tid == 0) f.tile_cnt[tile] = 0;
    __threadfence();
    __syncthreads();
    if (tid == 0) s_flag = (atomicAdd(&ctl->wave_ctas_done, 1) == ntiles - 1);
    __syncthreads();
    if (!s_flag) return;
    __threadfence();
    wave_finalize(f, it, s_red);
}

// ------------------------------------------------------------------ host launchers
template <class T>
static cudaError_t launch_wave(const Fit& f, int it, int grid, cudaStream_t st) {
    const size_t smem = pair_smem_bytes<T>();
    cudaError_t e = ensure_smem_attr(reinterpret_cast<const void*>(k_pair_wave<T>), smem);
    if (e != cudaSuccess) return e;
    k_pair_wave<T><<<grid, kPairThreads, smem, st>>>(f, it);
    return cudaGetLastError();
}

cudaError_t launch_pair_wave(const Fit& f, int it, int grid, cudaStream_t st) {
    return f.precision == LINGAM_MIXED ? launch_wave<float>(f, it, grid, st) : launch_wave<double>(f, it, grid, st);
}

}  // namespace lingam

"""The mixed path (FP32 pair measure, FP64 covariance downdates) on the inputs that push
its arithmetic hardest, against the FP64 oracle on the same FP32 values, in forced-order
mode so that every iteration is compared:

  - heavy tails: a variable whose normalised samples reach close to the largest value a
    normalised sample can take, sqrt(n - 1) (Samuelson's inequality), so that the
    exponentials e^{-2|u|} and e^{-u^2/2} flush to zero and the 32-sample products of
    (1 + e^{-2|u|}) mix factors of 2 and of 1;
  - near-collinear pairs: 1 - rho^2 just above the mixed path's degeneracy cut-off 2^-20,
    where the residual (x_i - rho x_j) / sqrt(1 - rho^2) amplifies the FP32 rounding of
    the rows about a thousandfold;
  - long rows: p = 50 with n = 10^5 and 10^6 samples, where the FP32 moment sums of a pair
    run over many 32-sample groups and many CTAs' partial slots.

Each test prints the largest score error it measured; the bound is the mixed path's
stated tolerance, 1e-4 absolute.
"""
import numpy as np
import pytest

import oracle
from paper_2109_13993_gb300 import lingam, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2109_13993_gb300 import build
    build.build()
    lingam.load()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _dev(X):
    return torch.tensor(np.ascontiguousarray(X), dtype=torch.float32, device="cuda")


def _forced_vs_oracle(X32, prune):
    """Forced along the oracle's order: (max |dS| over all complete scores, oracle order,
    GPU result).  Unpruned runs must have exactly the oracle's score layout."""
    o_order, o_B, o_S = oracle.fit(X32.astype(np.float64))
    res = lingam.fit(_dev(X32), precision="mixed", prune=prune, forced_order=o_order, want_scores=True)
    m = ~np.isnan(res.scores)
    assert not np.any(m & np.isnan(o_S))
    if not prune:
        assert np.array_equal(m, ~np.isnan(o_S))
    err = np.abs(res.scores[m] - o_S[m])
    scale = max(1.0, np.abs(o_B).max())
    eB = np.abs(res.B - o_B).max() / scale
    return float(err.max()), eB, o_order, res


@pytest.mark.parametrize("prune", [False, True])
def test_heavy_tailed_samples_near_the_samuelson_bound(prune):
    n = 4000
    d = synth.lingam_dataset(12, n, 0.3, seed=21)
    X = d.X.copy()
    sd5 = X[5].std()
    X[5, 100] += 2.0e4 * sd5            # one sample dominates row 5's variance
    sd8 = X[8].std()
    X[8, [7, 1500, 3001]] += np.array([40.0, -35.0, 30.0]) * sd8   # three outliers in row 8
    X32 = X.astype(np.float32)
    z5 = (X32[5].astype(np.float64) - X32[5].mean()) / X32[5].astype(np.float64).std(ddof=1)
    assert np.abs(z5).max() > 0.99 * np.sqrt(n - 1)
    err, eB, _, _ = _forced_vs_oracle(X32, prune)
    print(f"heavy tails (max |u| {np.abs(z5).max():.2f} of sqrt(n-1) = {np.sqrt(n - 1):.2f}), prune={prune}: "
          f"max |dS| {err:.2e}, B error {eB:.1e}")
    assert err <= TOL and eB <= TOL


@pytest.mark.parametrize("c", [1.5, 3.0])
def test_near_collinear_pair_just_above_the_cutoff(c):
    n = 5000
    d = synth.lingam_dataset(10, n, 0.3, seed=22)
    X = d.X.copy()
    e = synth.noise(synth.Stream(22, 5), synth.NOISE_LAPLACE, n)
    eps = np.sqrt(c * 2.0 ** -20)
    X[9] = X[2] + eps * X[2].std() * e
    X32 = X.astype(np.float32)
    rho = np.corrcoef(X32.astype(np.float64))[2, 9]
    om = 1.0 - rho * rho
    assert 2.0 ** -20 < om < 4.0 * 2.0 ** -20
    err, eB, _, _ = _forced_vs_oracle(X32, prune=False)
    # B: least squares on a predecessor set that holds the collinear pair has condition
    # number kappa of about 2 / (1 - rho^2); the mixed path's covariance carries the FP32
    # rounding of the normalised rows (about 1e-8, see test_gpu_gram.py), so B is known to
    # kappa x 1e-8 relative, not to the 1e-4 that holds for well-conditioned fits
    kappa = np.linalg.cond(np.corrcoef(X32.astype(np.float64)))
    print(f"near-collinear pair, 1 - rho^2 = {om / 2.0 ** -20:.2f} x 2^-20: max |dS| {err:.2e}, B error {eB:.1e} "
          f"(condition number {kappa:.1e})")
    assert err <= TOL
    assert eB <= max(TOL, kappa * 1e-8)


def test_long_rows_n_1e5():
    d = synth.lingam_dataset(50, 100_000, 4.0 / 49.0, seed=23)
    err, eB, _, _ = _forced_vs_oracle(d.X.astype(np.float32), prune=False)
    print(f"p=50, n=1e5: max |dS| {err:.2e}, B error {eB:.1e}")
    assert err <= TOL and eB <= TOL


def test_long_rows_n_1e6_first_iterations():
    """n = 10^6: the oracle's scores of iterations 0 and 1 (every remaining variable)
    against the GPU forced along the oracle's first two roots."""
    n = 1_000_000
    d = synth.lingam_dataset(50, n, 4.0 / 49.0, seed=24)
    X32 = d.X.astype(np.float32)
    X64 = X32.astype(np.float64)
    S0 = oracle.variable_scores(X64, np.zeros(0, dtype=np.int32), np.arange(50))
    r0 = int(np.lexsort((np.arange(50), S0))[0])
    alive1 = np.array([v for v in range(50) if v != r0])
    S1 = oracle.variable_scores(X64, np.array([r0]), alive1)
    r1 = int(alive1[np.lexsort((alive1, S1))[0]])
    forced = [r0, r1] + [v for v in range(50) if v not in (r0, r1)]
    res = lingam.fit(_dev(X32), precision="mixed", prune=False, forced_order=forced, want_scores=True, max_iters=2)
    e0 = np.abs(res.scores[0] - S0).max()
    e1 = np.abs(res.scores[1][alive1] - S1).max()
    assert np.all(np.isnan(res.scores[1][[r0]]))
    print(f"p=50, n=1e6: max |dS| iteration 0 {e0:.2e}, iteration 1 {e1:.2e}")
    assert e0 <= TOL and e1 <= TOL


def test_extreme_row_scales():
    """Rows scaled over 10^-30 ... 3 x 10^30 (all FP32-representable): NormalizeData of the
    FP32 copy runs in float-float arithmetic for rows whose magnitudes lie in [2^-60, 2^60]
    (its squared deviations scaled by an exact power of two) and in FP64 outside, so that
    neither overflows nor underflows.  Forced along the oracle's order, every score is within
    the tolerance and B, brought back to unit scales, within 1e-4."""
    d = synth.lingam_dataset(8, 2000, 0.4, seed=11)
    scales = np.array([1e25, 1e-25, 1e15, 1.0, 1e-15, 3e30, 1e-30, 7.0])
    X32 = (d.X * scales[:, None]).astype(np.float32)
    assert np.all(np.isfinite(X32)) and np.all(np.abs(X32[X32 != 0]) > 1e-37)
    o_order, o_B, o_S = oracle.fit(X32.astype(np.float64))
    res = lingam.fit(_dev(X32), precision="mixed", prune=False, forced_order=o_order, want_scores=True)
    m = ~np.isnan(res.scores)
    assert np.array_equal(m, ~np.isnan(o_S))
    err = float(np.abs(res.scores[m] - o_S[m]).max())
    unit = scales[None, :] / scales[:, None]   # B_ij s_j / s_i: the coefficients at unit scales
    eB = float(np.abs(res.B * unit - o_B * unit).max()) / max(1.0, float(np.abs(o_B * unit).max()))
    print(f"row scales 1e-30 .. 3e30: max |dS| {err:.2e}, B (unit scales) {eB:.2e}")
    assert err <= TOL
    assert eB <= 1e-4

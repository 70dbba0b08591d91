"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Each test ties one part of the oracle to something other than the oracle
itself: the worked example of the paper, closed forms, quadrature of the
expectations in Eq. HApp, invariances of the method, or a library routine for
a step (least squares).  A plausible mistake anywhere in the oracle (a
dropped term, a wrong sign or index, a transposed operand, a missing centring)
fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

from paper_2109_13993_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_fig1():
    lines = [ln.strip() for ln in open(os.path.join(GOLDEN, "fig1_sem.txt")) if ln.strip() and not ln.startswith("#")]
    b_at = lines.index("B")
    o_at = lines.index("ORDER_1BASED")
    B = np.array([[float(v) for v in ln.split()] for ln in lines[b_at + 1:o_at]])
    order = np.array([int(v) for v in lines[o_at + 1].split()]) - 1
    return B, order


# ---------------------------------------------------------------- constants (Eq. HApp)

def test_constants_are_the_printed_values(oracle_mod):
    c = oracle_mod.constants()
    assert c["k1"] == 79.047 and c["k2"] == 7.4129 and c["beta"] == 0.37457
    assert c["h_gauss"] == pytest.approx(0.5 * (1.0 + math.log(2.0 * math.pi)), rel=0, abs=1e-15)


def test_beta_is_gaussian_expectation_of_log_cosh():
    # beta = E[log cosh Z], Z ~ N(0,1), to the printed rounding.
    val, _ = integrate.quad(lambda z: math.log(math.cosh(z)) * math.exp(-z * z / 2) / math.sqrt(2 * math.pi),
                            -40, 40, limit=200)
    assert abs(val - 0.37457) < 5e-6


def test_k2_closed_form():
    # k2 = 36 / (8 sqrt(3) - 9) in the entropy approximation of Hyvarinen (1998).
    assert abs(36.0 / (8.0 * math.sqrt(3.0) - 9.0) - 7.4129) < 5e-5


def _quantile_sample(ppf, n):
    q = (np.arange(n) + 0.5) / n
    return ppf(q)


def test_entropy_vanishes_for_gaussian(oracle_mod):
    # For normalised Gaussian data both bracketed terms of Eq. HApp vanish,
    # so H(u) -> H(nu).  A deterministic quantile sample makes the sample
    # expectations accurate to O(1/n).
    u = oracle_mod.standardize(_quantile_sample(special.ndtri, 1_000_000))
    h = oracle_mod.entropy(u)
    assert abs(h - oracle_mod.constants()["h_gauss"]) < 2e-6


def _expected_entropy(lc, g, c):
    return c["h_gauss"] - c["k1"] * (lc - c["beta"]) ** 2 - c["k2"] * g ** 2


def test_entropy_uniform_by_quadrature(oracle_mod):
    c = oracle_mod.constants()
    a = math.sqrt(3.0)
    lc, _ = integrate.quad(lambda u: math.log(math.cosh(u)) / (2 * a), -a, a)
    u = oracle_mod.standardize(_quantile_sample(lambda q: -a + 2 * a * q, 1_000_000))
    assert oracle_mod.entropy(u) == pytest.approx(_expected_entropy(lc, 0.0, c), abs=2e-6)
    # the correction is far from zero for this non-Gaussian law
    assert c["h_gauss"] - oracle_mod.entropy(u) > 0.05


def test_entropy_skewed_by_quadrature(oracle_mod):
    # Exponential(1) shifted to mean 0: exercises the k2 term (odd moment).
    c = oracle_mod.constants()
    lc, _ = integrate.quad(lambda x: math.log(math.cosh(x - 1.0)) * math.exp(-x), 0, 60, limit=200)
    g, _ = integrate.quad(lambda x: (x - 1.0) * math.exp(-(x - 1.0) ** 2 / 2) * math.exp(-x), 0, 60, limit=200)
    assert abs(g) > 0.05
    u = oracle_mod.standardize(_quantile_sample(lambda q: -np.log1p(-q), 2_000_000))
    assert oracle_mod.entropy(u) == pytest.approx(_expected_entropy(lc, g, c), abs=2e-4)


# ---------------------------------------------------------------- pair measure (Eq. Itest)

def _two_var(n, seed, b=0.8):
    x1 = synth.noise(synth.Stream(seed, 11), synth.NOISE_UNIFORM, n)
    e = synth.noise(synth.Stream(seed, 12), synth.NOISE_LAPLACE, n)
    return x1, b * x1 + e


def test_pair_measure_antisymmetric(oracle_mod):
    x1, x2 = _two_var(20000, 3)
    a = oracle_mod.pair_measure(x1, x2)
    b = oracle_mod.pair_measure(x2, x1)
    assert a == pytest.approx(-b, rel=1e-12, abs=1e-15)


def test_pair_measure_points_from_cause_to_effect(oracle_mod):
    # I > 0 means x_i is the more independent (exogenous) of the two.
    for seed in (1, 2, 3):
        x1, x2 = _two_var(100_000, seed)
        assert oracle_mod.pair_measure(x1, x2) > 0
        order, _, S = oracle_mod.fit(np.stack([x1, x2]))
        assert list(order) == [0, 1]
        assert S[0, 0] == 0.0                      # min(0, I)^2 with I > 0
        I = oracle_mod.pair_measure(x1, x2)
        assert S[0, 1] == pytest.approx(I * I, rel=1e-12)
        order2, _, _ = oracle_mod.fit(np.stack([x2, x1]))
        assert list(order2) == [1, 0]


def test_pair_measure_matches_lstsq_route(oracle_mod):
    # Same measure with the regression step done by numpy's least squares
    # (with intercept) and normalisation by numpy's std(ddof=1).
    x1, x2 = _two_var(5000, 7)
    c = oracle_mod.constants()

    def norm(v):
        return (v - v.mean()) / v.std(ddof=1)

    def H(u):
        return _expected_entropy(np.mean(np.log(np.cosh(u))), np.mean(u * np.exp(-u * u / 2)), c)

    z1, z2 = norm(x1), norm(x2)
    A2 = np.stack([z2, np.ones_like(z2)], 1)
    A1 = np.stack([z1, np.ones_like(z1)], 1)
    r1 = z1 - A2 @ np.linalg.lstsq(A2, z1, rcond=None)[0]
    r2 = z2 - A1 @ np.linalg.lstsq(A1, z2, rcond=None)[0]
    expect = H(z2) + H(norm(r1)) - H(z1) - H(norm(r2))
    assert oracle_mod.pair_measure(x1, x2) == pytest.approx(expect, rel=1e-9, abs=1e-13)


def test_gaussian_pair_is_undecided(oracle_mod):
    s = synth.Stream(5, 1)
    z1 = s.normal(200_000)
    z2 = 0.6 * z1 + 0.8 * s.normal(200_000)
    x1n, _ = _two_var(200_000, 5, b=0.0)
    assert abs(oracle_mod.pair_measure(z1, z2)) < 1e-3 * abs(oracle_mod.pair_measure(x1n, 0.6 * x1n + z2))


# ---------------------------------------------------------------- closed forms (Sec. III-E)

def test_residual_variance_closed_form(oracle_mod):
    d = synth.workload("p20_n2000", seed=2)
    zi = oracle_mod.standardize(d.X[3])
    zj = oracle_mod.standardize(d.X[7])
    n = zi.size
    rho = float(zi @ zj) / (n - 1)
    r = oracle_mod.regress(zi, zj)
    assert r.mean() == pytest.approx(0.0, abs=1e-12)
    assert r.var(ddof=1) == pytest.approx(1.0 - rho * rho, rel=1e-12)     # Eq. var_update
    # Algorithm 7: the normalised residual is (x_w - Sigma[w,root] x_root) / sqrt(1 - Sigma^2)
    assert np.allclose(oracle_mod.standardize(r), (zi - rho * zj) / math.sqrt(1 - rho * rho), rtol=0, atol=1e-12)


def test_covariance_matrix_is_the_correlation_matrix(oracle_mod):
    # CalculateCovMat (Algorithm 3) on normalised rows is the sample correlation
    # matrix, whatever divisor the normalisation uses: numpy's corrcoef fixes it
    d = synth.workload("p20_n2000", seed=3)
    S = oracle_mod.covariance(d.X)
    C = np.corrcoef(d.X)
    assert S.shape == (20, 20)
    assert np.abs(S - C).max() < 1e-12
    assert np.abs(np.diag(S) - 1.0).max() < 1e-12
    # a row subset gives the matching sub-block (rows are normalised one by one)
    sub = [4, 11, 17]
    assert np.abs(oracle_mod.covariance(d.X[sub]) - S[np.ix_(sub, sub)]).max() < 1e-14


def test_covariance_update_closed_form(oracle_mod):
    d = synth.workload("p20_n2000", seed=4)
    z = [oracle_mod.standardize(d.X[k]) for k in (1, 5, 9)]
    n = z[0].size
    S = np.array([[float(a @ b) / (n - 1) for b in z] for a in z])
    ri = oracle_mod.regress(z[0], z[2])
    rj = oracle_mod.regress(z[1], z[2])
    cov = float((ri - ri.mean()) @ (rj - rj.mean())) / (n - 1)
    assert cov == pytest.approx(S[0, 1] - S[0, 2] * S[1, 2], rel=1e-12)     # Eq. CovUpdate
    corr = cov / (ri.std(ddof=1) * rj.std(ddof=1))
    assert corr == pytest.approx((S[0, 1] - S[0, 2] * S[1, 2]) /
                                 math.sqrt((1 - S[0, 2] ** 2) * (1 - S[1, 2] ** 2)), rel=1e-12)   # Algorithm 8


# ---------------------------------------------------------------- whole order (Algorithm 1)

def test_fig1_worked_example_order(oracle_mod):
    B_paper, order_paper = _read_fig1()
    d = synth.fig1_sem(100_000, seed=1)
    assert np.array_equal(d.B, B_paper)
    order, B, _ = oracle_mod.fit(d.X)
    assert list(order) == list(order_paper)
    assert np.max(np.abs(B - B_paper)) < 0.05
    P = B[np.ix_(order, order)]
    assert np.all(np.triu(P) == 0.0)


def _hamiltonian_dag(p, seed, n):
    s = synth.Stream(seed, 500 + p)
    pi = s.permutation(p)
    B = np.zeros((p, p))
    for k in range(1, p):
        for m in range(k):
            if m == k - 1 or s.uniform(1)[0] < 0.3:
                w = 0.5 + s.uniform(1)[0]
                B[pi[k], pi[m]] = w if s.uniform(1)[0] < 0.5 else -w
    X = np.zeros((p, n))
    for k in range(p):
        v = pi[k]
        kind = synth.NOISE_UNIFORM if s.uniform(1)[0] < 0.5 else synth.NOISE_LAPLACE
        X[v] = synth.noise(synth.Stream(seed, 600 + v), kind, n) + B[v] @ X
    return X, B, pi


@pytest.mark.parametrize("p,seed", [(3, 1), (4, 2), (5, 3), (6, 4), (6, 5)])
def test_tiny_dag_with_hamiltonian_path_recovers_unique_order(oracle_mod, p, seed):
    X, B_true, pi = _hamiltonian_dag(p, seed, 100_000)
    order, B, _ = oracle_mod.fit(X)
    assert list(order) == list(pi)
    assert np.max(np.abs(B - B_true)) < 0.05


def test_forced_order_reproduces_free_run(oracle_mod):
    d = synth.workload("p20_n2000", seed=3)
    order, B, S = oracle_mod.fit(d.X)
    order2, B2, S2 = oracle_mod.fit(d.X, forced_order=order)
    assert np.array_equal(order, order2)
    assert np.array_equal(np.isnan(S), np.isnan(S2))
    assert np.array_equal(S[~np.isnan(S)], S2[~np.isnan(S2)])
    # forcing another order leaves the first iteration's scores unchanged
    other = order[::-1].copy()
    order3, _, S3 = oracle_mod.fit(d.X, forced_order=other)
    assert np.array_equal(order3, other)
    assert np.array_equal(S3[0], S[0])


def test_scores_per_iteration_layout(oracle_mod):
    d = synth.workload("p20_n2000", seed=1)
    order, _, S = oracle_mod.fit(d.X)
    p = len(order)
    for it in range(p):
        removed = set(order[:it].tolist())
        for v in range(p):
            assert np.isnan(S[it, v]) == (v in removed)
        alive = [v for v in range(p) if v not in removed]
        best = min(alive, key=lambda v: (S[it, v], v))
        assert order[it] == best
    assert S[p - 1, order[p - 1]] == 0.0


def test_find_root_scores_matches_fit_first_iteration(oracle_mod):
    d = synth.workload("p20_n2000", seed=5)
    _, _, S = oracle_mod.fit(d.X, want_B=False)
    S0 = oracle_mod.find_root_scores(d.X, np.arange(20))
    assert np.array_equal(S0, S[0])


# ---------------------------------------------------------------- invariances

def test_affine_rescaling_leaves_result_unchanged(oracle_mod):
    d = synth.workload("p20_n2000", seed=6)
    s = synth.Stream(6, 3)
    a = 0.1 + 10 * s.uniform(20)
    c = 100 * (s.uniform(20) - 0.5)
    order, B, S = oracle_mod.fit(d.X)
    order2, B2, S2 = oracle_mod.fit(a[:, None] * d.X + c[:, None])
    assert np.array_equal(order, order2)
    m = ~np.isnan(S)
    assert np.allclose(S2[m], S[m], rtol=1e-9, atol=1e-15)
    # B is in the units of X: b_ij scales by a_i / a_j
    assert np.allclose(B2, B * a[:, None] / a[None, :], rtol=1e-8, atol=1e-12)


def test_relabelling_variables_permutes_the_result(oracle_mod):
    d = synth.workload("p20_n2000", seed=7)
    perm = synth.Stream(7, 9).permutation(20)
    inv = np.argsort(perm)
    order, B, S = oracle_mod.fit(d.X)
    order2, B2, S2 = oracle_mod.fit(d.X[perm])
    assert list(order2) == list(inv[order])
    m = ~np.isnan(S)
    assert np.allclose(S2[:, inv][m], S[m], rtol=1e-10, atol=1e-16)
    assert np.allclose(B2, B[np.ix_(perm, perm)], rtol=1e-10, atol=1e-13)


# ---------------------------------------------------------------- B (ordinary least squares on predecessors)

def test_B_is_least_squares_on_predecessors(oracle_mod):
    d = synth.workload("p20_n2000", seed=8)
    order, B, _ = oracle_mod.fit(d.X)
    Xc = d.X - d.X.mean(axis=1, keepdims=True)
    for k in range(1, 20):
        tgt, pred = order[k], order[:k]
        coef = np.linalg.lstsq(Xc[pred].T, Xc[tgt], rcond=None)[0]
        assert np.allclose(B[tgt, pred], coef, rtol=1e-9, atol=1e-11)
        resid = Xc[tgt] - B[tgt] @ Xc
        assert np.max(np.abs(Xc[pred] @ resid)) < 1e-8 * np.linalg.norm(Xc[tgt]) * np.sqrt(d.X.shape[1])
    assert np.all(np.triu(B[np.ix_(order, order)]) == 0.0)


# ---------------------------------------------------------------- edge cases

def test_single_variable(oracle_mod):
    x = synth.noise(synth.Stream(1, 1), synth.NOISE_UNIFORM, 100)[None, :]
    order, B, S = oracle_mod.fit(x)
    assert list(order) == [0] and B.shape == (1, 1) and B[0, 0] == 0.0 and S[0, 0] == 0.0


def test_constant_row_is_degenerate(oracle_mod):
    d = synth.workload("p20_n2000", seed=1)
    X = d.X.copy()
    X[4] = 3.0
    with pytest.raises(RuntimeError) as e:
        oracle_mod.fit(X)
    assert e.value.status == -2


def test_generator_is_deterministic():
    a = synth.workload("p20_n2000", seed=9)
    b = synth.workload("p20_n2000", seed=9)
    c = synth.workload("p20_n2000", seed=10)
    assert np.array_equal(a.X, b.X) and np.array_equal(a.B, b.B)
    assert not np.array_equal(a.X, c.X)
    P = a.B[np.ix_(a.order, a.order)]
    assert np.all(np.triu(P) == 0.0)


def test_variable_scores_match_fit(oracle_mod):
    d = synth.workload("p20_n2000", seed=2)
    order, _, S = oracle_mod.fit(d.X, want_B=False)
    for k in (0, 3, 11):
        alive = [v for v in range(20) if v not in set(order[:k].tolist())]
        vs = alive[::3]
        got = oracle_mod.variable_scores(d.X, order[:k], vs)
        assert np.allclose(got, S[k, vs], rtol=1e-12, atol=1e-18)


# ---------------------------------------------------------------- brute force on p <= 6 (Algorithms 1-2)

# The printed constants of Eq. HApp, typed here again so that this check shares no value
# with the oracle's source.
_K1, _K2, _BETA = 79.047, 7.4129, 0.37457
_H_NU = 0.5 * (1.0 + math.log(2.0 * math.pi))


def _naive_directlingam(X, prior=None):
    """DirectLiNGAM written out directly in numpy, with no intermediate reuse: at every
    iteration, for every ordered pair (i, j) of the remaining variables, both rows are
    normalised (mean, sample sd with divisor n - 1), each is regressed on the other
    (slope = sample covariance / sample variance, np.cov), both residuals normalised,
    I = H(x_j) + H(r_i) - H(x_i) - H(r_j) (Eq. Itest with Eq. HApp) and
    S_i += min(0, I)^2 (Algorithm 2); the root is the argmin, lowest index on ties; every
    remaining row is then regressed on the root's row (RegressRoot, Algorithm 1).
    Returns the order and the p x p score matrix (NaN for removed variables)."""
    W = np.array(X, dtype=np.float64)
    p = W.shape[0]

    def norm(v):
        return (v - v.mean()) / v.std(ddof=1)

    def H(u):
        return _H_NU - _K1 * (np.mean(np.log(np.cosh(u))) - _BETA) ** 2 - _K2 * np.mean(u * np.exp(-u * u / 2)) ** 2

    U = list(range(p))
    order, S_all = [], np.full((p, p), np.nan)
    for it in range(p):
        # with prior knowledge only variables without a known ancestor left in U may be the root
        cand = [i for i in U if prior is None or not any(prior[i, j] == 1 for j in U if j != i)]
        for i in cand:
            s = 0.0
            for j in U:
                if j == i:
                    continue
                xi, xj = norm(W[i]), norm(W[j])
                c = np.cov(xi, xj)
                ri = norm(xi - c[0, 1] / c[1, 1] * xj)
                rj = norm(xj - c[0, 1] / c[0, 0] * xi)
                I = H(xj) + H(ri) - H(xi) - H(rj)
                s += min(0.0, I) ** 2
            S_all[it, i] = s
        root = min(cand, key=lambda v: (S_all[it, v], v))
        order.append(root)
        U.remove(root)
        for w in U:
            c = np.cov(W[w], W[root])
            W[w] = W[w] - c[0, 1] / c[1, 1] * W[root]
    return np.array(order), S_all


_BRUTE_CASES = [(3, 2000, 11), (4, 3000, 12), (5, 4000, 13), (6, 5000, 14), (6, 2500, 15)]


@pytest.mark.parametrize("p,n,seed", _BRUTE_CASES)
def test_every_score_of_every_iteration_by_brute_force(oracle_mod, p, n, seed):
    """Brute-force pin: on seeded p <= 6 DAGs every S_i of every iteration, recomputed by the
    naive formula above, equals the oracle's within 1e-12 (absolute), and so does the order."""
    d = synth.lingam_dataset(p, n, 0.6, seed=seed)
    order_b, S_b = _naive_directlingam(d.X)
    order_o, _, S_o = oracle_mod.fit(d.X, want_B=False)
    assert list(order_o) == list(order_b)
    m = ~np.isnan(S_b)
    assert np.array_equal(m, ~np.isnan(S_o))
    assert np.max(np.abs(S_o[m] - S_b[m])) <= 1e-12
    assert np.all(S_b[m] >= 0.0)
    assert np.max(S_b[m]) > 1e-6          # the case exercises non-trivial scores


# ---------------------------------------------------------------- prior knowledge (known ancestors)

def _prior_from_order(order, p, pairs):
    """prior[i, j] = 1 for the given (earlier, later) position pairs of `order`: x_j a known
    ancestor of x_i; everything else unknown (-1)."""
    prior = -np.ones((p, p), dtype=np.int8)
    for a, b in pairs:
        prior[order[b], order[a]] = 1
    return prior


def test_prior_knowledge_of_a_total_order_forces_it(oracle_mod):
    # a chain of known ancestors through all variables leaves exactly one root candidate per
    # iteration, so the order is the chain whatever the data say (here the reverse of the
    # data's own order)
    d = synth.workload("p20_n2000", seed=4)
    free, _, _ = oracle_mod.fit(d.X, want_B=False)
    chain = free[::-1].copy()
    prior = _prior_from_order(chain, 20, [(k, k + 1) for k in range(19)])
    order, _, S = oracle_mod.fit(d.X, want_B=False, prior=prior)
    assert list(order) == list(chain)
    for it in range(20):
        assert np.count_nonzero(~np.isnan(S[it])) == 1


@pytest.mark.parametrize("p,n,seed", _BRUTE_CASES)
def test_prior_knowledge_by_brute_force(oracle_mod, p, n, seed):
    # a random partial prior consistent with a random order: the naive restatement with the
    # same candidate rule gives the same scores (NaN for non-candidates) and order
    d = synth.lingam_dataset(p, n, 0.6, seed=seed)
    s = synth.Stream(seed, 77)
    perm = s.permutation(p)
    pairs = [(a, b) for a in range(p) for b in range(a + 1, p) if s.uniform(1)[0] < 0.4]
    prior = _prior_from_order(perm, p, pairs)
    order_b, S_b = _naive_directlingam(d.X, prior)
    order_o, _, S_o = oracle_mod.fit(d.X, want_B=False, prior=prior)
    assert list(order_o) == list(order_b)
    m = ~np.isnan(S_b)
    assert np.array_equal(m, ~np.isnan(S_o))
    assert np.max(np.abs(S_o[m] - S_b[m])) <= 1e-12
    pos = {v: k for k, v in enumerate(order_o)}
    for i in range(p):
        for j in range(p):
            if prior[i, j] == 1:
                assert pos[j] < pos[i]          # every known ancestor comes first


def test_cyclic_prior_is_rejected(oracle_mod):
    d = synth.workload("p20_n2000", seed=1)
    prior = -np.ones((20, 20), dtype=np.int8)
    prior[3, 7] = prior[7, 11] = prior[11, 3] = 1
    with pytest.raises(RuntimeError) as e:
        oracle_mod.fit(d.X, prior=prior)
    assert e.value.status == -1

"""Batches through lingam_fit_batch and lingam_fit_bootstrap: many independent
problems in one persistent launch (and, from the second call on the same
workspace and shapes, from a captured CUDA graph).

A problem's result in a batch differs from its single fit only in how its
pairs' samples are grouped into partial sums (the stream-K partition spans all
problems), i.e. in FP32 rounding.  So orders must agree with the single fit (or
the oracle) on every iteration the reference's margin resolves, and may differ
after the first unresolved one.  The per-score bound of the mixed path is
tau = kappa sqrt(m S) + m (2e-6)^2 with kappa = 1e-5 (the bound asserted by the
single-fit parity tests, which measure about 2e-6).
"""
import numpy as np
import pytest

import oracle
from paper_2109_13993_gb300 import lingam, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KAPPA = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2109_13993_gb300 import build
    build.build()
    lingam.load()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _dev(X, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(X), dtype=dtype, device="cuda")


def _tau(S, m):
    return KAPPA * np.sqrt(max(m, 1) * max(S, 0.0)) + max(m, 1) * (2e-6) ** 2


def _agree_until_unresolved(order, ref_order, ref_root, ref_margin):
    """The orders agree up to their first difference, and that iteration's reference
    margin is within the two scores' bounds (a resolved iteration never differs).
    Returns the length of the common prefix."""
    p = len(ref_order)
    for it in range(p):
        if order[it] != ref_order[it]:
            m = p - it - 1
            tau1 = _tau(ref_root[it], m)
            tau2 = _tau(ref_root[it] + ref_margin[it], m)
            assert not ref_margin[it] > tau1 + tau2, f"resolved iteration {it} differs"
            return it
    return p


def _single(X):
    """Reference single fit with complete scores (no pruning): exact roots and margins."""
    r = lingam.fit(X, precision="mixed", prune=False, want_scores=True)
    roots, margins = _oracle_margins(r.scores)
    return r, roots, margins


def _oracle_margins(S):
    roots, margins = [], []
    for row in S:
        v = np.sort(row[~np.isnan(row)])
        roots.append(v[0])
        margins.append(v[1] - v[0] if len(v) > 1 else np.inf)
    return np.array(roots), np.array(margins)


def test_batch_matches_single_fits():
    ds = synth.uneven_batch(6, seed=4)
    Xs = [_dev(d.X[:, : min(d.X.shape[1], 3000)].astype(np.float32)) for d in ds]
    res = lingam.fit_batch(Xs, precision="mixed")
    assert res.status == 0 and np.all(res.statuses == 0)
    for X, o, B in zip(Xs, res.orders, res.Bs):
        single, roots, margins = _single(X)
        k = _agree_until_unresolved(o, single.order, roots, margins)
        print(f"p={X.shape[0]} n={X.shape[1]}: batch order equals the single fit on {k} of {len(o)} iterations")
        if k == len(o):
            assert np.abs(B - single.B).max() <= 1e-6 * max(1.0, np.abs(single.B).max())


def _member_vs_oracle(order, scores, root_score, margin_lb, o_order, o_S, atol, rtol=0.0):
    """A batch member against the oracle, element by element.  The member and the oracle
    start every iteration in the same state until their roots first differ (iteration k),
    so at iterations 0..k every score the member completed is within atol + rtol |S| of the
    oracle's, its root's score is the oracle's score of that root within the same bound,
    and its margin lower bound does not exceed the oracle's margin by more than twice it.
    The first difference must be an iteration whose oracle margin is within 2 tau (tau =
    the largest error measured at that iteration, at least 2e-7 on the mixed path), so the
    order is the oracle's whenever every margin is resolved.  Returns (k, max error)."""
    p = len(o_order)
    diff = np.nonzero(np.asarray(order) != np.asarray(o_order))[0]
    k = int(diff[0]) if len(diff) else p
    worst = 0.0
    for it in range(min(k + 1, p)):
        row, ora = scores[it], o_S[it]
        complete = ~np.isnan(row)
        assert not np.any(complete & np.isnan(ora)), f"iteration {it}: a removed variable has a score"
        assert complete[order[it]], f"iteration {it}: the root's score is incomplete"
        err = np.abs(row[complete] - ora[complete])
        bound = atol + rtol * np.abs(ora[complete])
        assert np.all(err <= bound), f"iteration {it}: max |dS| {err.max():.3e}"
        assert abs(root_score[it] - ora[order[it]]) <= atol + rtol * abs(ora[order[it]])
        worst = max(worst, float(err.max()))
        alive = np.sort(ora[~np.isnan(ora)])
        if len(alive) > 1:
            tau = max(float(err.max()), 2e-7 if rtol == 0.0 else 1e-10 * alive[0])
            true_margin = alive[1] - alive[0]
            assert margin_lb[it] <= true_margin + 2 * (atol + rtol * alive[1])
            if it == k:
                assert true_margin <= 2 * tau, f"resolved iteration {it} differs"
    return k, worst


def _hard_members(rng_seed):
    """A heavy-tailed member (one sample near the largest normalised value sqrt(n - 1)) and a
    near-collinear member (1 - rho^2 = 2 x 2^-20 between two of its variables)."""
    d = synth.lingam_dataset(10, 3000, 0.3, seed=rng_seed)
    Xh = d.X.copy()
    Xh[4, 10] += 1.0e4 * Xh[4].std()
    d2 = synth.lingam_dataset(8, 3000, 0.3, seed=rng_seed + 1)
    Xc = d2.X.copy()
    e = synth.noise(synth.Stream(rng_seed, 5), synth.NOISE_UNIFORM, 3000)
    Xc[7] = Xc[1] + np.sqrt(2.0 * 2.0 ** -20) * Xc[1].std() * e
    return [Xh.astype(np.float32), Xc.astype(np.float32)]


@pytest.mark.parametrize("tile_i,tile_j", [(0, 0), (64, 32), (32, 32), (64, 16), (32, 16), (1, 1)])
def test_batch_matches_oracle(tile_i, tile_j):
    """Batch members (uneven sizes, one above 64 variables, plus a heavy-tailed and a
    near-collinear member) against the oracle, with each pair-tile shape of the batch kernel
    (0 x 0: the batch autotuner's untuned default, the pair mode below 129 variables): every
    complete score, root score and margin bound of every iteration on the common prefix
    within 1e-4, and the full order wherever every margin is resolved."""
    sizes = [(5, 4000), (12, 3000), (20, 2000), (33, 2500), (70, 1500)]
    ds = []
    for k, (p, n) in enumerate(sizes):
        ds.append(synth.lingam_dataset(p, n, min(1.0, 4.0 / (p - 1)), seed=40 + k).X.astype(np.float32))
    ds += _hard_members(48)
    res = lingam.fit_batch([_dev(X) for X in ds], precision="mixed", want_report=True, want_scores=True,
                           tile_i=tile_i, tile_j=tile_j)
    assert res.status == 0
    for m, (X32, o, B) in enumerate(zip(ds, res.orders, res.Bs)):
        o_order, o_B, o_S = oracle.fit(X32.astype(np.float64))
        k, worst = _member_vs_oracle(o, res.scores[m], res.root_scores[m], res.margins[m], o_order, o_S, atol=1e-4)
        print(f"tiles {tile_i}x{tile_j} member {m} (p={X32.shape[0]}): order equals the oracle on {k} of {len(o)} "
              f"iterations, max |dS| {worst:.2e} on the common prefix")
        if k == len(o):
            assert np.abs(B - o_B).max() <= 1e-4 * max(1.0, np.abs(o_B).max())


def test_batch_fp64_matches_oracle():
    """FP64 batch members against the oracle: scores and root scores within 1e-10 relative
    (floor 1e-14) on the common prefix, B within 1e-10 when the whole order agrees."""
    sizes = [(6, 2000), (15, 1500)]
    data = [synth.lingam_dataset(p, n, 0.4, seed=60 + k).X for k, (p, n) in enumerate(sizes)]
    res = lingam.fit_batch([_dev(X, torch.float64) for X in data], precision="fp64", want_report=True,
                           want_scores=True)
    assert res.status == 0
    for m, (X, o, B) in enumerate(zip(data, res.orders, res.Bs)):
        o_order, o_B, o_S = oracle.fit(X)
        k, worst = _member_vs_oracle(o, res.scores[m], res.root_scores[m], res.margins[m], o_order, o_S,
                                     atol=1e-14, rtol=1e-10)
        print(f"FP64 member {m}: order equals the oracle on {k} of {len(o)} iterations, max |dS| {worst:.2e}")
        if k == len(o):
            assert np.abs(B - o_B).max() <= 1e-10 * max(1.0, np.abs(o_B).max())


def test_bootstrap_matches_gathered_single_fits():
    d = synth.lingam_dataset(20, 1500, 0.2, seed=8)
    X = d.X.astype(np.float32)
    idx = synth.bootstrap_indices(1500, 8, seed=3)
    assert idx.min() >= 0 and idx.max() < 1500
    res = lingam.fit_bootstrap(_dev(X), idx, precision="mixed")
    assert res.status == 0 and np.all(res.statuses == 0)
    for b in range(8):
        Xb = np.ascontiguousarray(X[:, idx[b]])
        single, roots, margins = _single(_dev(Xb))
        k = _agree_until_unresolved(res.orders[b], single.order, roots, margins)
        print(f"bootstrap {b}: order equals the gathered single fit on {k} of 20 iterations")
    # two resamples against the oracle on the gathered data, element by element
    rs = lingam.fit_bootstrap(_dev(X), idx, precision="mixed", want_report=True, want_scores=True)
    assert all(np.array_equal(a, b) for a, b in zip(res.orders, rs.orders))
    for b in (0, 5):
        Xb = X[:, idx[b]].astype(np.float64)
        o_order, o_B, o_S = oracle.fit(Xb)
        k, worst = _member_vs_oracle(rs.orders[b], rs.scores[b], rs.root_scores[b], rs.margins[b], o_order, o_S,
                                     atol=1e-4)
        print(f"bootstrap {b} vs oracle: order equal on {k} of 20 iterations, max |dS| {worst:.2e}")
    # host indices and device indices give the same result; reports carry every
    # resample's evaluated pairs (at most all unordered pairs of each iteration)
    res2 = lingam.fit_bootstrap(_dev(X), torch.tensor(idx, device="cuda"), precision="mixed", want_report=True)
    assert all(np.array_equal(a, b) for a, b in zip(res.orders, res2.orders))
    assert len(res2.pairs) == 8
    for pp in res2.pairs:
        r = 20 - np.arange(20)
        assert np.all(pp >= 0) and np.all(pp <= r * (r - 1) // 2) and pp[0] > 0


def test_batch_edge_sizes():
    """Tiny and ragged members in one batch (p = 1, 2, 3 and tile-edge sizes, n down to 3):
    every member succeeds and agrees with its single fit; p = 1 and 2 give the trivial
    orders' structure (a permutation)."""
    sizes = [(1, 50), (2, 3), (3, 5), (17, 257), (33, 1000), (65, 400), (2, 700)]
    ds = [synth.lingam_dataset(p, n, min(1.0, 4.0 / max(p - 1, 1)), seed=90 + k).X.astype(np.float32)
          for k, (p, n) in enumerate(sizes)]
    Xs = [_dev(X) for X in ds]
    res = lingam.fit_batch(Xs, precision="mixed")
    assert res.status == 0 and np.all(res.statuses == 0)
    for X, (p, n), o, B in zip(Xs, sizes, res.orders, res.Bs):
        assert sorted(o.tolist()) == list(range(p))
        single, roots, margins = _single(X)
        k = _agree_until_unresolved(o, single.order, roots, margins)
        print(f"p={p} n={n}: batch order equals the single fit on {k} of {p} iterations")
        if k == p:
            assert np.abs(B - single.B).max() <= 1e-6 * max(1.0, np.abs(single.B).max())


def test_batch_gram_small_and_large_members():
    """Members on both sides of the batched small-problem covariance (p <= 128 in one launch,
    exact FP32 products in float-float sums; larger p on the tensor-core Gram): every member
    agrees with its single fit (tensor-core Gram) on the resolved prefix, and B within 1e-6
    where the whole order agrees."""
    sizes = [(3, 900), (50, 2000), (127, 1200), (128, 1100), (129, 1000), (140, 700)]
    ds = [synth.lingam_dataset(p, n, min(1.0, 4.0 / (p - 1)), seed=120 + k).X.astype(np.float32)
          for k, (p, n) in enumerate(sizes)]
    Xs = [_dev(X) for X in ds]
    res = lingam.fit_batch(Xs, precision="mixed", tile_i=1, tile_j=1)
    assert res.status == 0 and np.all(res.statuses == 0)
    for X, (p, n), o, B in zip(Xs, sizes, res.orders, res.Bs):
        single, roots, margins = _single(X)
        k = _agree_until_unresolved(o, single.order, roots, margins)
        print(f"p={p} n={n}: batch order equals the single fit on {k} of {p} iterations")
        if k == p:
            assert np.abs(B - single.B).max() <= 1e-6 * max(1.0, np.abs(single.B).max())


def test_batch_degenerate_member_does_not_stop_the_others():
    ds = [synth.lingam_dataset(10, 800, 0.3, seed=70 + k).X.astype(np.float32) for k in range(3)]
    ds[1][4] = 2.5   # a constant row
    res = lingam.fit_batch([_dev(X) for X in ds], precision="mixed")
    assert res.status == lingam.LINGAM_EDEGENERATE
    assert list(res.statuses) == [0, lingam.LINGAM_EDEGENERATE, 0]
    for k in (0, 2):
        single, roots, margins = _single(_dev(ds[k]))
        assert _agree_until_unresolved(res.orders[k], single.order, roots, margins) > 0


def test_batch_graph_replay_is_identical():
    ds = synth.uneven_batch(5, seed=9)
    Xs = [_dev(d.X[:, :2000].astype(np.float32)) for d in ds]
    ws = lingam.batch_workspace([X.shape[0] for X in Xs], [X.shape[1] for X in Xs])
    runs = [lingam.fit_batch(Xs, precision="mixed", workspace=ws) for _ in range(3)]   # eager, capture, replay
    for r in runs[1:]:
        assert r.status == 0
        assert all(np.array_equal(a, b) for a, b in zip(runs[0].orders, r.orders))
        assert all(np.array_equal(a, b) for a, b in zip(runs[0].Bs, r.Bs))
    # new data of the same shapes through the replayed graph
    ds2 = synth.uneven_batch(5, seed=9)
    Xs2 = [_dev(np.ascontiguousarray(d.X[:, :2000][::-1]).astype(np.float32)) for d in ds2]
    r2 = lingam.fit_batch(Xs2, precision="mixed", workspace=ws)
    for X, o in zip(Xs2, r2.orders):
        single, roots, margins = _single(X)
        _agree_until_unresolved(o, single.order, roots, margins)


def test_batched_workload_full_size():
    """256 bootstrap resamples of one p=50, n=2000 dataset and 64 uneven datasets
    (p in 20..120, n in 500..8000), mixed path: every problem succeeds and sampled
    problems agree with their single fits."""
    d = synth.lingam_dataset(50, 2000, 4.0 / 49.0, seed=5)
    X = d.X.astype(np.float32)
    idx = synth.bootstrap_indices(2000, 256, seed=6)
    rb = lingam.fit_bootstrap(_dev(X), idx, precision="mixed")
    assert rb.status == 0 and np.all(rb.statuses == 0)
    for b in (0, 97, 255):
        single, roots, margins = _single(_dev(np.ascontiguousarray(X[:, idx[b]])))
        k = _agree_until_unresolved(rb.orders[b], single.order, roots, margins)
        print(f"bootstrap resample {b}: order equals the single fit on {k} of 50 iterations")
    ds = synth.uneven_batch(64, seed=7)
    Xs = [_dev(dd.X.astype(np.float32)) for dd in ds]
    ru = lingam.fit_batch(Xs, precision="mixed")
    assert ru.status == 0 and np.all(ru.statuses == 0)
    for k in (0, 31, 63):
        single, roots, margins = _single(Xs[k])
        j = _agree_until_unresolved(ru.orders[k], single.order, roots, margins)
        print(f"uneven dataset {k} (p={Xs[k].shape[0]}): order equals the single fit on {j} iterations")


def test_batch_autotuner_records_its_choice():
    """lingam_autotune_batch times the three tile shapes on the caller's batch and records the
    fastest for the bucket of the largest p and n; later calls with tile_i = tile_j = 0 use it
    and give orders within the batch's own tolerance of an explicit-shape call."""
    ds = synth.uneven_batch(12, seed=21)
    Xs = [_dev(d.X[:, : min(d.X.shape[1], 2000)].astype(np.float32)) for d in ds]
    maxp = max(x.shape[0] for x in Xs)
    maxn = max(x.shape[1] for x in Xs)
    untuned = (1, 1) if maxp <= 128 else (32, 32)
    lingam.autotune_reset()
    assert lingam.batch_tile_shape(maxp, maxn) == untuned
    shape, ms = lingam.autotune_batch(Xs)
    print(f"batch autotune (12 datasets, p <= {maxp}, n <= {maxn}): {ms} -> {shape}")
    assert shape in ms and all(v > 0 for v in ms.values())
    assert ms[shape] == min(ms.values())
    assert lingam.batch_tile_shape(maxp, maxn) == shape
    auto = lingam.fit_batch(Xs, precision="mixed")
    expl = lingam.fit_batch(Xs, precision="mixed", tile_i=shape[0], tile_j=shape[1])
    assert auto.status == 0 and all(np.array_equal(a, b) for a, b in zip(auto.orders, expl.orders))
    lingam.autotune_reset()
    assert lingam.batch_tile_shape(maxp, maxn) == untuned

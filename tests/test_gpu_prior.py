"""Prior knowledge (known ancestors) through lingam_fit against the oracle's fit with the
same prior: at every iteration only variables with no known ancestor left may be the root,
every remaining variable is still a partner, and the scores of the others are NaN on both
sides.  The paper notes that DirectLiNGAM accepts prior knowledge (Sec. II-C) without
defining it; the reading (known ancestors restrict the root candidates) is the oracle's."""
import numpy as np
import pytest

import oracle
from paper_2109_13993_gb300 import lingam, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2109_13993_gb300 import build
    build.build()
    lingam.load()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _prior(order, frac, seed):
    """Known ancestors consistent with `order`: each (earlier, later) pair with probability frac."""
    p = len(order)
    s = synth.Stream(seed, 88)
    prior = -np.ones((p, p), dtype=np.int8)
    for a in range(p):
        u = s.uniform(p)
        for b in range(a + 1, p):
            if u[b] < frac:
                prior[order[b], order[a]] = 1
    return prior


@pytest.mark.parametrize("name,precision,frac", [("p20_n2000", "fp64", 0.3), ("p20_n2000", "mixed", 0.3),
                                                 ("p100_n10000", "mixed", 0.05)])
def test_prior_knowledge_matches_oracle(name, precision, frac):
    d = synth.workload(name, seed=2)
    p = d.X.shape[0]
    # a prior drawn from a random order (not the data's), so that it changes the result
    perm = synth.Stream(5, 9).permutation(p)
    prior = _prior(perm, frac, seed=3)
    X = d.X if precision == "fp64" else d.X.astype(np.float32)
    o_order, o_B, o_S = oracle.fit(X.astype(np.float64), prior=prior)
    dt = torch.float64 if precision == "fp64" else torch.float32
    Xd = torch.tensor(X, dtype=dt, device="cuda")
    res = lingam.fit(Xd, precision=precision, forced_order=o_order, want_scores=True, prior=prior)
    tol = (1e-10, 1e-14) if precision == "fp64" else (0.0, 1e-4)
    done = 0
    for it in range(p):
        row, ora = res.scores[it], o_S[it]
        comp = ~np.isnan(row)
        assert not np.any(comp & np.isnan(ora)), f"iteration {it}: a non-candidate has a score"
        err = np.abs(row[comp] - ora[comp])
        assert np.all(err <= tol[0] * np.abs(ora[comp]) + tol[1]), f"iteration {it}: {err.max():.3e}"
        done += int(comp.sum())
    free = lingam.fit(Xd, precision=precision, prior=prior)
    pos = {int(v): k for k, v in enumerate(free.order)}
    for i in range(p):
        for j in range(p):
            if prior[i, j] == 1:
                assert pos[j] < pos[i], f"known ancestor {j} of {i} ordered after it"
    agree = int(np.argmax(free.order != o_order)) if np.any(free.order != o_order) else p
    print(f"{name} {precision}: {done} complete scores checked, free run equal to the oracle on the first {agree} "
          f"iterations, every known ancestor first")
    if precision == "fp64":
        assert agree == p


def test_prior_of_a_total_order_forces_it():
    d = synth.workload("p100_n10000", seed=4)
    X = torch.tensor(d.X.astype(np.float32), device="cuda")
    chain = synth.Stream(4, 2).permutation(100)
    prior = -np.ones((100, 100), dtype=np.int8)
    for k in range(99):
        prior[chain[k + 1], chain[k]] = 1
    res = lingam.fit(X, prior=prior, want_scores=True)
    assert list(res.order) == list(chain)
    assert all(np.count_nonzero(~np.isnan(res.scores[it])) == 1 for it in range(100))

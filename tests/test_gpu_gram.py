"""Parity of CalculateCovMat (Algorithm 3) through lingam_covariance with the
FP64 CPU oracle's covariance of the normalised rows.

Tolerances.  FP64 path: 1e-12 absolute (|Sigma| <= 1, FP64 sums of n terms).
Mixed path: the tensor-core product of the FP32 normalised rows is error-free
up to about 2^-24 (exact integer digit products, float-float drains, FP64
split sums), so the error is that of rounding the normalised rows to FP32:
each element moves by at most 2^-24 of itself, which moves Sigma_ij by at most
2^-23 sum_t |x_i x_j| / (n-1) <= 2^-23 n/(n-1).  The bound used is that plus
2^-24; the measured errors sit one to two orders of magnitude below it.  The
diagonal is exactly 1 and the matrix exactly symmetric on both paths.
"""
import numpy as np
import pytest

import oracle
from paper_2109_13993_gb300 import lingam, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL_FP64 = 1e-12


def tol_mixed(n):
    return 2.0 ** -23 * n / (n - 1) + 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2109_13993_gb300 import build
    build.build()
    lingam.load()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _data(p, n, seed):
    if p >= 2:
        d = synth.lingam_dataset(p, n, edge_prob=min(1.0, 4.0 / max(1, p - 1)), seed=seed)
        return d.X
    return synth.Stream(seed, 7).normal(n).reshape(1, n)


def _check(S, ref, tol):
    assert S.shape == ref.shape
    assert np.array_equal(np.diag(S), np.ones(S.shape[0])), "diagonal is not exactly 1"
    assert np.array_equal(S, S.T), "not exactly symmetric"
    off = ~np.eye(S.shape[0], dtype=bool)
    err = np.abs(S - ref)[off].max() if off.any() else 0.0
    assert err <= tol, f"max off-diagonal error {err:.3e} > {tol:.1e}"
    return err


# sizes: one partial tile; two tiles with ragged rows; several tiles and a
# ragged sample tail; a sample count that is not a multiple of 32; tiny cases
CASES = [(20, 2000), (129, 1000), (300, 5000), (257, 4097), (2, 3), (1, 10), (5, 33)]


@pytest.mark.parametrize("p,n", CASES)
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_covariance_matches_oracle(p, n, precision):
    X = _data(p, n, seed=p * 7 + n)
    if precision == "mixed":
        X = X.astype(np.float32).astype(np.float64)   # both sides see the same FP32 rows
    ref = oracle.covariance(X)
    Xd = torch.tensor(X, dtype=torch.float32 if precision == "mixed" else torch.float64, device="cuda")
    S, info = lingam.covariance(Xd, precision=precision)
    err = _check(S, ref, tol_mixed(n) if precision == "mixed" else TOL_FP64)
    print(f"p={p} n={n} {precision}: max err {err:.3e}, gram {info['gram']:.3f} ms")


def test_covariance_host_input_and_float64_rows():
    X = _data(100, 3000, seed=5)
    X32 = X.astype(np.float32)
    S1, _ = lingam.covariance(X32, precision="mixed")                            # host FP32 rows
    S2, _ = lingam.covariance(torch.tensor(X, device="cuda"), precision="mixed")  # device FP64 rows
    _check(S1, oracle.covariance(X32.astype(np.float64)), tol_mixed(3000))
    _check(S2, oracle.covariance(X), tol_mixed(3000))


def test_covariance_full_size_sampled_rows():
    # p = 1000, n = 1e4 (the benchmark's workload): the oracle covers a sample of
    # 48 rows, whose covariance block does not depend on the other rows
    d = synth.workload("p1000_n10000", seed=1)
    Xd = torch.tensor(d.X, dtype=torch.float32, device="cuda")
    S, info = lingam.covariance(Xd, precision="mixed")
    rows = np.sort(synth.Stream(3, 11).permutation(1000)[:48])
    ref = oracle.covariance(d.X[rows].astype(np.float32).astype(np.float64))
    err = _check(S[np.ix_(rows, rows)], ref, tol_mixed(10000))
    assert np.array_equal(S, S.T)
    print(f"p=1000 n=1e4 mixed: sampled max err {err:.3e}, gram {info['gram']:.3f} ms")


def test_covariance_degenerate_row():
    X = _data(40, 500, seed=9)
    X[17] = 3.0
    with pytest.raises(lingam.LingamError) as e:
        lingam.covariance(torch.tensor(X, dtype=torch.float32, device="cuda"), precision="mixed")
    assert e.value.status == lingam.LINGAM_EDEGENERATE


def test_covariance_repeated_calls_are_identical():
    X = torch.tensor(_data(200, 6000, seed=4), dtype=torch.float32, device="cuda")
    ws = lingam.alloc_workspace(lingam.workspace_size(200, 6000, "mixed"))
    S1, _ = lingam.covariance(X, precision="mixed", workspace=ws)
    S2, _ = lingam.covariance(X, precision="mixed", workspace=ws)
    assert np.array_equal(S1, S2)

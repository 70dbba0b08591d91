"""Seeded synthetic LiNGAM data: inputs for the CUDA path, the oracle and the bench.

This module only draws input data; it holds none of the ordering method's
arithmetic.  Every random number comes from SplitMix64 (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014), written out
here as a counter-based stream: the k-th draw of a stream keyed by (seed, tag)
is mix(key + (k + 1) * GOLDEN).  The same seed gives the same data on every
machine up to the last bit of the libm calls used by the inverse transforms.

Model (Sec. II-B, Eq. base_mat): X = B X + N with B strictly lower triangular
in a causal order, i.e. X = (I - B)^{-1} N.  Data are returned row-major
p x n (row i = the n samples of variable X_i).

Generator recipe (identical for every workload, sizes vary):
  1. a random permutation pi gives the causal order;
  2. B is strictly lower triangular in pi-order, each edge present with
     probability q;
  3. edge weights are uniform on [-1.5, -0.5] U [0.5, 1.5];
  4. each variable draws its noise type: uniform(-sqrt3, sqrt3),
     Laplace(0, 1/sqrt2), or sign(z)|z|^e with z ~ N(0,1), e ~ U[1.2, 2.0];
  5. X = (I - B)^{-1} N, solved in causal order in float64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


class Stream:
    """Counter-based SplitMix64 stream keyed by (seed, tag)."""

    def __init__(self, seed: int, tag: int):
        seed, tag = int(seed), int(tag)
        with np.errstate(over="ignore"):
            k = np.array([(seed * 0x100000001B3 + tag * 0x2545F4914F6CDD1D) & 0xFFFFFFFFFFFFFFFF],
                         dtype=np.uint64)
            self.key = _mix(k)[0]
        self.counter = 0

    def u64(self, count: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            idx = np.arange(self.counter + 1, self.counter + 1 + count, dtype=np.uint64)
            z = self.key + idx * _GOLDEN
            out = _mix(z)
        self.counter += count
        return out

    def uniform(self, count: int) -> np.ndarray:
        """Doubles in the open interval (0, 1)."""
        return ((self.u64(count) >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)

    def normal(self, count: int) -> np.ndarray:
        """Box-Muller transform of two uniforms per draw."""
        u1 = self.uniform(count)
        u2 = self.uniform(count)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)

    def integers(self, low: int, high: int, count: int) -> np.ndarray:
        """Uniform integers in [low, high] (inclusive)."""
        span = high - low + 1
        return low + np.minimum((self.uniform(count) * span).astype(np.int64), span - 1)

    def permutation(self, m: int) -> np.ndarray:
        return np.argsort(self.uniform(m), kind="stable")


NOISE_UNIFORM, NOISE_LAPLACE, NOISE_POWER = 0, 1, 2


def noise(stream: Stream, kind: int, n: int) -> np.ndarray:
    if kind == NOISE_UNIFORM:
        return (2.0 * stream.uniform(n) - 1.0) * math.sqrt(3.0)
    if kind == NOISE_LAPLACE:
        u = stream.uniform(n) - 0.5
        return -(1.0 / math.sqrt(2.0)) * np.sign(u) * np.log1p(-2.0 * np.abs(u))
    if kind == NOISE_POWER:
        e = 1.2 + 0.8 * stream.uniform(1)[0]
        z = stream.normal(n)
        return np.sign(z) * np.abs(z) ** e
    raise ValueError(kind)


@dataclass
class Dataset:
    X: np.ndarray          # p x n float64, row-major
    B: np.ndarray          # p x p true weights, B[i, j] = effect of X_j on X_i
    order: np.ndarray      # a true causal order (0-based variable indices)
    noise_kind: np.ndarray  # per-variable noise family


def lingam_dataset(p: int, n: int, edge_prob: float, seed: int,
                   noise_kinds: tuple[int, ...] = (NOISE_UNIFORM, NOISE_LAPLACE, NOISE_POWER)) -> Dataset:
    """Random LiNGAM data set following the recipe in the module docstring."""
    s_perm = Stream(seed, 1)
    s_edge = Stream(seed, 2)
    s_w = Stream(seed, 3)
    s_kind = Stream(seed, 4)
    pi = s_perm.permutation(p)
    B = np.zeros((p, p))
    if p > 1:
        tri = np.tril_indices(p, -1)            # (a, b) with a > b in causal positions
        present = s_edge.uniform(len(tri[0])) < edge_prob
        mag = 0.5 + s_w.uniform(len(tri[0]))
        sgn = np.where(s_w.uniform(len(tri[0])) < 0.5, -1.0, 1.0)
        w = np.where(present, sgn * mag, 0.0)
        B[pi[tri[0]], pi[tri[1]]] = w
    kinds = np.array(noise_kinds)[s_kind.integers(0, len(noise_kinds) - 1, p)]
    E = np.empty((p, n))
    for v in range(p):
        E[v] = noise(Stream(seed, 1000 + v), int(kinds[v]), n)
    X = np.empty((p, n))
    for k in range(p):            # solve (I - B) X = E in causal order
        v = pi[k]
        parents = np.nonzero(B[v])[0]
        X[v] = E[v] + (B[v, parents] @ X[parents] if len(parents) else 0.0)
    return Dataset(X=X, B=B, order=pi.astype(np.int64), noise_kind=kinds)


def fig1_sem(n: int, seed: int) -> Dataset:
    """The worked example SEM of Fig. 1 (Eq. sem, Eq. base_mat_ex), 0-based.

    X3 = N3, X5 = 5 X3 + N5, X1 = 3 X5 + N1, X4 = 4 X1 + N4, X2 = 6 X3 - 3 X4 + N2,
    with uniform noises of unit variance.  Its causal order [3,5,1,4,2]
    (1-based) is unique since 3 -> 5 -> 1 -> 4 -> 2 is a Hamiltonian path.
    """
    B = np.zeros((5, 5))
    B[0, 4] = 3.0
    B[1, 2] = 6.0
    B[1, 3] = -3.0
    B[3, 0] = 4.0
    B[4, 2] = 5.0
    order = np.array([2, 4, 0, 3, 1])
    E = np.stack([noise(Stream(seed, 1000 + v), NOISE_UNIFORM, n) for v in range(5)])
    X = np.zeros((5, n))
    for v in order:               # parents are computed before their children
        X[v] = E[v] + B[v] @ X
    return Dataset(X=X, B=B, order=order, noise_kind=np.zeros(5, dtype=np.int64))


def scalability_dataset(p: int, n: int, dense: bool, seed: int) -> Dataset:
    """The synthetic graphs of the paper's scalability experiment (Sec. V-D).

    Every variable draws its number of parents uniformly from [1, 0.2 p] (sparse) or
    [0.25 p, 0.5 p] (dense), capped by the number of variables before it in a random causal
    order, and takes them uniformly among those; each edge weight is uniform in
    [-0.95, -0.5] U [0.5, 0.95] (the paper prints the negative interval reversed); each
    noise is Gaussian passed through sign(z)|z|^q with q uniform in [0.5, 0.8] U [1.2, 2].
    Samples are generated recursively in causal order.  The paper does not say how it
    keeps the variances finite (with 250-500 parents of weight up to 0.95 they overflow
    within a few hundred variables); here every variable is scaled to unit sample variance
    right after it is generated, which rescales its row of B and its noise and leaves the
    causal structure as it is (B is returned for the scaled variables)."""
    s_perm, s_cnt, s_par, s_w, s_q = (Stream(seed, t) for t in (21, 22, 23, 24, 25))
    pi = s_perm.permutation(p)
    lo, hi = (max(1, int(math.ceil(0.25 * p))), max(1, int(0.5 * p))) if dense else (1, max(1, int(0.2 * p)))
    counts = s_cnt.integers(lo, hi, p)
    B = np.zeros((p, p))
    X = np.empty((p, n))
    for k in range(p):
        v = pi[k]
        m = min(int(counts[k]), k)
        z = Stream(seed, 3000 + v).normal(n)
        u = s_q.uniform(2)
        q = 0.5 + 0.3 * u[1] if u[0] < 0.5 else 1.2 + 0.8 * u[1]
        x = np.sign(z) * np.abs(z) ** q
        if m > 0:
            par = pi[:k][np.argsort(s_par.uniform(k), kind="stable")[:m]]
            w = (0.5 + 0.45 * s_w.uniform(m)) * np.where(s_w.uniform(m) < 0.5, -1.0, 1.0)
            B[v, par] = w
            x = x + w @ X[par]
        sd = x.std(ddof=1)
        X[v] = x / sd
        B[v] /= sd
    return Dataset(X=X, B=B, order=pi.astype(np.int64), noise_kind=np.full(p, NOISE_POWER))


def bootstrap_indices(n: int, count: int, seed: int) -> np.ndarray:
    """count x n observation indices drawn with replacement (one row per resample)."""
    s = Stream(seed, 77)
    return s.integers(0, n - 1, count * n).reshape(count, n).astype(np.int32)


# Workloads of the paper-derived benchmark configurations.  Names state sizes.
def workload(name: str, seed: int = 1) -> Dataset:
    if name == "p20_n2000":
        return lingam_dataset(20, 2000, 3.0 / 19.0, seed)
    if name == "p100_n10000":
        return lingam_dataset(100, 10000, 4.0 / 99.0, seed)
    if name == "p300_n5000":
        return lingam_dataset(300, 5000, 6.0 / 299.0, seed)
    if name == "p1000_n10000":
        return lingam_dataset(1000, 10000, 4.0 / 999.0, seed)
    raise KeyError(name)


def uneven_batch(count: int, seed: int) -> list[Dataset]:
    """count independent datasets, p uniform in {20..120}, n uniform in {500..8000}."""
    s = Stream(seed, 99)
    ps = s.integers(20, 120, count)
    ns = s.integers(500, 8000, count)
    return [lingam_dataset(int(p), int(n), 4.0 / max(int(p) - 1, 1), seed * 1000 + 7 + k)
            for k, (p, n) in enumerate(zip(ps, ns))]

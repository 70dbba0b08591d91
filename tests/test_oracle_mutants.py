"""Plants plausible mistakes in copies of the oracle (CPU only) and checks that
the pin tests catch every one of them.

Each mutant is the oracle's C source with one textual change, built into a
temporary library; the pin tests of test_oracle_pins.py then run against it
and at least one must fail.
"""
import ctypes
import os
import subprocess
import tempfile

import pytest

import oracle
from oracle import oracle as omod
import tests.test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(omod.__file__), "lingam_oracle.c")

MUTANTS = {
    "drop_k2_term": ("- ORACLE_K2 * g * g", ""),
    "beta_sign": ("double a = lc - ORACLE_BETA;", "double a = lc + ORACLE_BETA;"),
    "gauss_kernel_exponent": ("exp(-u[t] * u[t] / 2.0)", "exp(-u[t] * u[t])"),
    "transposed_I": ("double I = hj + oracle_entropy(ri, n) - hi - oracle_entropy(rj, n);",
                     "double I = hi + oracle_entropy(ri, n) - hj - oracle_entropy(rj, n);"),
    "swapped_residual": ("if ((st = oracle_regress(xi, xj, n, ri)) != ORACLE_OK) return st;",
                         "if ((st = oracle_regress(xj, xi, n, ri)) != ORACLE_OK) return st;"),
    "score_keeps_positive_part": ("double m = I < 0.0 ? I : 0.0;", "double m = I > 0.0 ? I : 0.0;"),
    "score_not_squared": ("s += m * m;", "s += -m;"),
    "argmax_root": ("else if (S[a] < S[best] || (S[a] == S[best] && U[a] < U[best])) best = a;",
                    "else if (S[a] > S[best] || (S[a] == S[best] && U[a] < U[best])) best = a;"),
    "no_centring_in_cov": ("for (long t = 0; t < n; ++t) s += (x[t] - mx) * (y[t] - my);",
                           "for (long t = 0; t < n; ++t) s += x[t] * y[t];"),
    "variance_divisor_n": ("v /= (double)(n - 1);", "v /= (double)n;"),
    "regress_root_backwards": ("st = oracle_regress(W + (size_t)w * n, W + (size_t)root * n, n, tmp);",
                               "st = oracle_regress(W + (size_t)root * n, W + (size_t)w * n, n, tmp);"),
    "no_regress_root": ("if (st == ORACLE_OK) memcpy(W + (size_t)w * n, tmp, sizeof(double) * (size_t)n);",
                        "(void)tmp;"),
    "covariance_wrong_operand": ("for (long t = 0; t < n; ++t) s += zi[t] * zj[t];",
                                 "for (long t = 0; t < n; ++t) s += zi[t] * zi[t];"),
    "covariance_divisor_n": ("out[(size_t)i * p + j] = s / (double)(n - 1);", "out[(size_t)i * p + j] = s / (double)n;"),
    "B_wrong_predecessor_index": ("for (int a = 0; a < k; ++a) B[(size_t)tgt * p + K[a]] = rhs[a];",
                                  "for (int a = 0; a < k; ++a) B[(size_t)tgt * p + a] = rhs[a];"),
    "B_transposed_store": ("for (int a = 0; a < k; ++a) B[(size_t)tgt * p + K[a]] = rhs[a];",
                           "for (int a = 0; a < k; ++a) B[(size_t)K[a] * p + tgt] = rhs[a];"),
    # a wrong partner set in FindRoot (Algorithm 2): the variable at position 0 of U is
    # never used as a partner
    "partner_set_drops_first": ("            if (b == a) continue;", "            if (b == a || b == 0) continue;"),
    # prior knowledge read transposed (x_i taken as the known ancestor of x_j)
    "prior_transposed": ("if (b != a && prior[(size_t)U[a] * p + U[b]] == 1) return 0;",
                         "if (b != a && prior[(size_t)U[b] * p + U[a]] == 1) return 0;"),
    # RegressRoot (Algorithm 1) skips the first remaining variable
    "regress_root_skips_first": ("for (int a = 0; a < r && st == ORACLE_OK; ++a) {\n            int w = U[a];",
                                 "for (int a = 1; a < r && st == ORACLE_OK; ++a) {\n            int w = U[a];"),
}

# Mutants that the brute-force pin (every score of every iteration on p <= 6) must catch
# by itself: the score definition, the partner set and the data update between iterations.
BRUTE_FORCE_MUTANTS = ("partner_set_drops_first", "regress_root_skips_first", "no_regress_root",
                       "regress_root_backwards", "score_keeps_positive_part", "score_not_squared",
                       "transposed_I", "swapped_residual", "drop_k2_term", "beta_sign", "gauss_kernel_exponent")


def _pin_calls():
    """(name, callable(view)) for every pin that takes the oracle as argument."""
    out = []
    for name in dir(pins):
        if not name.startswith("test_"):
            continue
        fn = getattr(pins, name)
        if "oracle_mod" not in fn.__code__.co_varnames[:fn.__code__.co_argcount]:
            continue
        marks = getattr(fn, "pytestmark", [])
        params = [m for m in marks if m.name == "parametrize"]
        if params:
            argnames = [a.strip() for a in params[0].args[0].split(",")]
            for vals in params[0].args[1]:
                kw = dict(zip(argnames, vals if isinstance(vals, tuple) else (vals,)))
                out.append((f"{name}{vals}", lambda v, fn=fn, kw=kw: fn(v, **kw)))
        else:
            out.append((name, lambda v, fn=fn: fn(v)))
    return out


@pytest.fixture(scope="module")
def tmpdir_mut():
    with tempfile.TemporaryDirectory() as d:
        yield d


def _mutant_view(mutant, tmpdir_mut):
    """The oracle with one planted mistake, built into a temporary library."""
    old, new = MUTANTS[mutant]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site of {mutant} not found"
    path_c = os.path.join(tmpdir_mut, f"{mutant}.c")
    path_so = os.path.join(tmpdir_mut, f"lib{mutant}.so")
    if not os.path.exists(path_so):
        open(path_c, "w").write(src.replace(old, new))
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-std=c11", "-D_GNU_SOURCE",
                               "-ffp-contract=off", "-o", path_so, path_c, "-lm"])
    return omod.View(omod.load(path_so))


@pytest.mark.parametrize("mutant", BRUTE_FORCE_MUTANTS)
def test_brute_force_pin_catches_mutant(mutant, tmpdir_mut):
    view = _mutant_view(mutant, tmpdir_mut)
    caught = False
    for case in pins._BRUTE_CASES:
        try:
            pins.test_every_score_of_every_iteration_by_brute_force(view, *case)
        except Exception:
            caught = True
            break
    assert caught, f"the brute-force pin missed mutant {mutant}"


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_catch_mutant(mutant, tmpdir_mut):
    view = _mutant_view(mutant, tmpdir_mut)
    caught = []
    for name, call in _pin_calls():
        try:
            call(view)
        except Exception:            # an assertion or an oracle error both count as caught
            caught.append(name)
            break
    assert caught, f"no pin caught mutant {mutant}"

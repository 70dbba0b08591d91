"""ctypes binding of oracle/lingam_oracle.c (test infrastructure only).

Every function follows the paper's DirectLiNGAM (Sec. II-C, Algorithms 1-2,
Eqs. Itest and HApp) in FP64 on the CPU; see the C source header for the
readings of the points the paper leaves open.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lingam_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD_DIR, "liblingam_oracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, EDEGENERATE, ENOMEM = 0, -1, -2, -3


class OracleError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"oracle {what} failed with status {status}")
        self.status = status


def lib_path() -> str:
    return _LIB


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, IEEE FP64, no fast-math)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-std=c11", "-D_GNU_SOURCE",
                               "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def load(path: str):
    """Load an oracle library built from lingam_oracle.c and declare its signatures."""
    L = ctypes.CDLL(path)
    _declare(L)
    return L


def _get():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = load(_LIB)
    return _lib


def _declare(L):
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    for name in ("oracle_const_k1", "oracle_const_k2", "oracle_const_beta", "oracle_const_h_gauss"):
        getattr(L, name).restype = ctypes.c_double
        getattr(L, name).argtypes = []
    L.oracle_standardize.argtypes = [dp, ctypes.c_long, dp]
    L.oracle_covariance.argtypes = [dp, ctypes.c_int, ctypes.c_long, dp]
    L.oracle_entropy.argtypes = [dp, ctypes.c_long]
    L.oracle_entropy.restype = ctypes.c_double
    L.oracle_regress.argtypes = [dp, dp, ctypes.c_long, dp]
    L.oracle_pair_measure.argtypes = [dp, dp, ctypes.c_long, dp]
    L.oracle_find_root_scores.argtypes = [dp, ctypes.c_int, ctypes.c_long, ip, ctypes.c_int, ctypes.c_int, dp]
    L.oracle_fit_B.argtypes = [dp, ctypes.c_int, ctypes.c_long, ip, dp]
    L.oracle_fit.argtypes = [dp, ctypes.c_int, ctypes.c_long, ip, dp, dp, ip, ctypes.c_int]
    L.oracle_fit_prior.argtypes = [dp, ctypes.c_int, ctypes.c_long, ctypes.POINTER(ctypes.c_byte), ip, dp, dp, ip,
                                   ctypes.c_int]
    L.oracle_pair_measures.argtypes = [dp, ctypes.c_long, ip, ip, ctypes.c_int, ctypes.c_int, dp]
    L.oracle_num_threads.argtypes = [ctypes.c_int]
    L.oracle_variable_scores.argtypes = [dp, ctypes.c_int, ctypes.c_long, ip, ctypes.c_int, ip, ctypes.c_int,
                                         ctypes.c_int, dp]


def _d(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _rows(X) -> np.ndarray:
    return np.ascontiguousarray(X, dtype=np.float64)


def constants(lib=None) -> dict:
    L = (lib or _get())
    return {"k1": L.oracle_const_k1(), "k2": L.oracle_const_k2(), "beta": L.oracle_const_beta(),
            "h_gauss": L.oracle_const_h_gauss()}


def num_threads(nthreads: int = 0, lib=None) -> int:
    return int((lib or _get()).oracle_num_threads(nthreads))


def standardize(x, lib=None) -> np.ndarray:
    x = _rows(x)
    out = np.empty_like(x)
    st = (lib or _get()).oracle_standardize(_d(x), x.size, _d(out))
    if st != OK:
        raise OracleError(st, "standardize")
    return out


def covariance(X, lib=None) -> np.ndarray:
    """CalculateCovMat (Algorithm 3): covariance of the normalised rows of X (p x n)."""
    X = _rows(X)
    p, n = X.shape
    out = np.empty((p, p))
    st = (lib or _get()).oracle_covariance(_d(X), p, n, _d(out))
    if st != OK:
        raise OracleError(st, "covariance")
    return out


def entropy(u, lib=None) -> float:
    """Eq. HApp on an already normalised sample."""
    u = _rows(u)
    return float((lib or _get()).oracle_entropy(_d(u), u.size))


def regress(x, y, lib=None) -> np.ndarray:
    x, y = _rows(x), _rows(y)
    r = np.empty_like(x)
    st = (lib or _get()).oracle_regress(_d(x), _d(y), x.size, _d(r))
    if st != OK:
        raise OracleError(st, "regress")
    return r


def pair_measure(xi, xj, lib=None) -> float:
    """I(x_i, x_j, r_i^(j), r_j^(i)) of Eq. Itest for raw rows."""
    xi, xj = _rows(xi), _rows(xj)
    out = np.zeros(1)
    st = (lib or _get()).oracle_pair_measure(_d(xi), _d(xj), xi.size, _d(out))
    if st != OK:
        raise OracleError(st, "pair_measure")
    return float(out[0])


def pair_measures(X, pairs, nthreads: int = 0, lib=None) -> np.ndarray:
    """I for each (i, j) in pairs, on raw rows of X (p x n)."""
    X = _rows(X)
    pairs = np.asarray(pairs, dtype=np.int32).reshape(-1, 2)
    pi = np.ascontiguousarray(pairs[:, 0])
    pj = np.ascontiguousarray(pairs[:, 1])
    out = np.zeros(len(pairs))
    st = (lib or _get()).oracle_pair_measures(_d(X), X.shape[1], _i(pi), _i(pj), len(pairs), nthreads, _d(out))
    if st != OK:
        raise OracleError(st, "pair_measures")
    return out


def find_root_scores(X, U, nthreads: int = 0, lib=None) -> np.ndarray:
    """Scores S (Alg. 2) of the variables U (by position in U) on raw rows X."""
    X = _rows(X)
    U = np.ascontiguousarray(U, dtype=np.int32)
    S = np.zeros(len(U))
    st = (lib or _get()).oracle_find_root_scores(_d(X), X.shape[0], X.shape[1], _i(U), len(U), nthreads, _d(S))
    if st != OK:
        raise OracleError(st, "find_root_scores")
    return S


def fit_B(X, order, lib=None) -> np.ndarray:
    X = _rows(X)
    K = np.ascontiguousarray(order, dtype=np.int32)
    p = X.shape[0]
    B = np.zeros((p, p))
    st = (lib or _get()).oracle_fit_B(_d(X), p, X.shape[1], _i(K), _d(B))
    if st != OK:
        raise OracleError(st, "fit_B")
    return B


def fit(X, forced_order=None, want_scores: bool = True, want_B: bool = True, nthreads: int = 0, lib=None,
        prior=None):
    """Algorithm 1.  Returns (order, B or None, scores p x p or None).  prior (p x p, values
    -1/0/1): prior[i, j] == 1 says x_j is a known ancestor of x_i; then only variables with
    no known ancestor left are root candidates, the others' scores are NaN."""
    X = _rows(X)
    p, n = X.shape
    order = np.zeros(p, dtype=np.int32)
    B = np.zeros((p, p)) if want_B else None
    S = np.full((p, p), np.nan) if want_scores else None
    forced = None if forced_order is None else np.ascontiguousarray(forced_order, dtype=np.int32)
    L = lib or _get()
    args = (_d(X), p, n)
    tail = (_i(order), _d(B) if B is not None else None, _d(S) if S is not None else None,
            _i(forced) if forced is not None else None, nthreads)
    if prior is None:
        st = L.oracle_fit(*args, *tail)
    else:
        pr = np.ascontiguousarray(prior, dtype=np.int8)
        st = L.oracle_fit_prior(*args, pr.ctypes.data_as(ctypes.POINTER(ctypes.c_byte)), *tail)
    if st != OK:
        raise OracleError(st, "fit")
    return order, B, S


def variable_scores(X, prefix, vars_, nthreads: int = 0, lib=None) -> np.ndarray:
    """S_v (Alg. 2) for each v in vars_, after the roots in prefix were removed (Alg. 1)."""
    X = _rows(X)
    pre = np.ascontiguousarray(prefix, dtype=np.int32)
    vs = np.ascontiguousarray(vars_, dtype=np.int32)
    out = np.zeros(len(vs))
    st = (lib or _get()).oracle_variable_scores(_d(X), X.shape[0], X.shape[1], _i(pre) if len(pre) else None,
                                                len(pre), _i(vs), len(vs), nthreads, _d(out))
    if st != OK:
        raise OracleError(st, "variable_scores")
    return out


class View:
    """The module's functions bound to one loaded oracle library (e.g. a test build)."""

    _names = ("constants", "num_threads", "standardize", "covariance", "entropy", "regress", "pair_measure", "pair_measures",
              "find_root_scores", "fit_B", "fit", "variable_scores")

    def __init__(self, lib):
        import functools
        g = globals()
        for name in self._names:
            setattr(self, name, functools.partial(g[name], lib=lib))

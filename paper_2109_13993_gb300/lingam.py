"""Python binding of the C ABI in include/lingam.h (argument marshalling only).

Every step of the ordering runs in the CUDA library liblingam_gb300.so; this
module only loads it, allocates the device workspace with PyTorch, and moves
arguments across the ABI.  There is no CPU fallback: if the library is not
built, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

LINGAM_OK, LINGAM_EINVAL, LINGAM_EDEGENERATE, LINGAM_ENOMEM, LINGAM_ECUDA, LINGAM_ETIMEOUT = 0, -1, -2, -3, -4, -5
LINGAM_EBOUNDS = -6
LINGAM_FP64, LINGAM_MIXED = 0, 1
LINGAM_F32, LINGAM_F64 = 0, 1

_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_dbl_p = ctypes.POINTER(ctypes.c_double)
_c_ll_p = ctypes.POINTER(ctypes.c_longlong)


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("input_dtype", ctypes.c_int), ("prune", ctypes.c_int),
                ("reuse", ctypes.c_int), ("tile_i", ctypes.c_int), ("tile_j", ctypes.c_int),
                ("split_n", ctypes.c_int), ("timeout_s", ctypes.c_double), ("stream", ctypes.c_void_p),
                ("forced_order", _c_int_p), ("max_iters", ctypes.c_int), ("timing", ctypes.c_int),
                ("prior", ctypes.c_void_p), ("gamma0", ctypes.c_double), ("gamma_c", ctypes.c_double)]


class Report(ctypes.Structure):
    _fields_ = [("root_score", _c_dbl_p), ("margin_lb", _c_dbl_p), ("pairs_evaluated", _c_ll_p),
                ("scores", _c_dbl_p), ("t_standardize_ms", ctypes.c_double), ("t_gram_ms", ctypes.c_double),
                ("t_order_ms", ctypes.c_double), ("t_B_ms", ctypes.c_double), ("pairs_total", ctypes.c_longlong),
                ("pairs_unpruned", ctypes.c_longlong), ("t_pair_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_longlong), ("t_pair_iter_ms", _c_dbl_p),
                ("t_compute_ms", ctypes.c_double), ("t_merge_ms", ctypes.c_double), ("t_remove_ms", ctypes.c_double),
                ("threshold_updates", ctypes.c_longlong), ("waves", ctypes.c_longlong),
                ("tile_pairs", ctypes.c_longlong), ("empty_col_pairs", ctypes.c_longlong),
                ("pad_row_pairs", ctypes.c_longlong)]


class LingamError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"lingam status {status}: {msg}")
        self.status = status


_lib = None


def lib_path() -> str:
    return _build.LIB


def load():
    """Load the CUDA library (raises if it has not been built).  The environment variable
    LINGAM_LIBRARY may name another build of it (e.g. build.DEBUG_LIB)."""
    global _lib
    if _lib is not None:
        return _lib
    path = os.environ.get("LINGAM_LIBRARY") or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(path)
    L.lingam_default_opts.argtypes = [ctypes.POINTER(Opts)]
    L.lingam_default_opts.restype = None
    L.lingam_workspace_size.argtypes = [ctypes.c_longlong, ctypes.c_longlong, ctypes.POINTER(Opts)]
    L.lingam_workspace_size.restype = ctypes.c_size_t
    L.lingam_fit.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p,
                             ctypes.c_void_p, ctypes.POINTER(Opts), ctypes.POINTER(Report)]
    L.lingam_fit.restype = ctypes.c_int
    L.lingam_workspace_size_batch.argtypes = [ctypes.c_int, _c_ll_p, _c_ll_p, ctypes.POINTER(Opts)]
    L.lingam_workspace_size_batch.restype = ctypes.c_size_t
    L.lingam_fit_batch.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p), _c_ll_p, _c_ll_p,
                                   ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p,
                                   ctypes.POINTER(Opts), _c_int_p, ctypes.POINTER(Report)]
    L.lingam_fit_batch.restype = ctypes.c_int
    L.lingam_workspace_size_bootstrap.argtypes = [ctypes.c_longlong, ctypes.c_longlong, ctypes.c_int,
                                                  ctypes.POINTER(Opts)]
    L.lingam_workspace_size_bootstrap.restype = ctypes.c_size_t
    L.lingam_fit_bootstrap.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_int,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.POINTER(Opts), _c_int_p, ctypes.POINTER(Report)]
    L.lingam_fit_bootstrap.restype = ctypes.c_int
    L.lingam_fit_static.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.POINTER(Opts), ctypes.POINTER(Report)]
    L.lingam_fit_static.restype = ctypes.c_int
    L.lingam_covariance.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.POINTER(Opts), ctypes.POINTER(Report)]
    L.lingam_covariance.restype = ctypes.c_int
    L.lingam_tile_rows.argtypes = [ctypes.c_longlong, ctypes.c_longlong]
    L.lingam_tile_rows.restype = ctypes.c_int
    L.lingam_tile_cols.argtypes = [ctypes.c_longlong, ctypes.c_longlong]
    L.lingam_tile_cols.restype = ctypes.c_int
    L.lingam_autotune.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_void_p,
                                  ctypes.POINTER(Opts), _c_int_p, _c_int_p, _c_dbl_p]
    L.lingam_autotune.restype = ctypes.c_int
    L.lingam_batch_tile_rows.argtypes = [ctypes.c_longlong, ctypes.c_longlong]
    L.lingam_batch_tile_rows.restype = ctypes.c_int
    L.lingam_batch_tile_cols.argtypes = [ctypes.c_longlong, ctypes.c_longlong]
    L.lingam_batch_tile_cols.restype = ctypes.c_int
    L.lingam_autotune_batch.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p), _c_ll_p, _c_ll_p,
                                        ctypes.c_void_p, ctypes.POINTER(Opts), _c_int_p, _c_int_p,
                                        ctypes.POINTER(ctypes.c_double)]
    L.lingam_autotune_batch.restype = ctypes.c_int
    L.lingam_autotune_reset.argtypes = []
    L.lingam_autotune_reset.restype = None
    L.lingam_status_string.argtypes = [ctypes.c_int]
    L.lingam_status_string.restype = ctypes.c_char_p
    L.lingam_selftest_wait.argtypes = [ctypes.c_int, ctypes.c_double, _c_int_p]
    L.lingam_selftest_wait.restype = ctypes.c_int
    _lib = L
    return L


def header_functions() -> list[str]:
    """Names of the functions declared in include/lingam.h."""
    hdr = open(os.path.join(_build.INCLUDE, "lingam.h")).read()
    return sorted(set(re.findall(r"\b(lingam_[a-z_0-9]+)\s*\(", hdr)))


def status_string(status: int) -> str:
    return load().lingam_status_string(status).decode()


def make_opts(precision: str = "mixed", input_dtype=np.float32, prune: bool = True, reuse: bool = True,
              split_n: int = 0, timeout_s: float = 10.0, stream=None, forced_order=None, max_iters: int = 0,
              timing: bool = False, tile_i: int = 0, tile_j: int = 0, prior=None, gamma0: float = 0.0,
              gamma_c: float = 2.0) -> tuple[Opts, object]:
    o = Opts()
    load().lingam_default_opts(ctypes.byref(o))
    o.precision = {"mixed": LINGAM_MIXED, "fp64": LINGAM_FP64}[precision]
    o.input_dtype = LINGAM_F32 if np.dtype(input_dtype) == np.float32 else LINGAM_F64
    o.prune = int(prune)
    o.reuse = int(reuse)
    o.split_n = int(split_n)
    o.timeout_s = float(timeout_s)
    o.stream = ctypes.c_void_p(stream) if stream else None
    o.max_iters = int(max_iters)
    o.timing = int(bool(timing))
    o.tile_i = int(tile_i)
    o.tile_j = int(tile_j)
    o.gamma0 = float(gamma0)
    o.gamma_c = float(gamma_c)
    keep = []
    if forced_order is not None:
        fo = np.ascontiguousarray(forced_order, dtype=np.int32)
        o.forced_order = fo.ctypes.data_as(_c_int_p)
        keep.append(fo)
    if prior is not None:
        pr = np.ascontiguousarray(prior, dtype=np.int8)
        o.prior = ctypes.c_void_p(pr.ctypes.data)
        keep.append(pr)
    return o, keep


def workspace_size(p: int, n: int, precision: str = "mixed", input_dtype=np.float32) -> int:
    o, _ = make_opts(precision, input_dtype)
    return int(load().lingam_workspace_size(p, n, ctypes.byref(o)))


@dataclass
class FitResult:
    order: np.ndarray
    B: np.ndarray | None
    root_score: np.ndarray
    margin_lb: np.ndarray
    pairs_evaluated: np.ndarray
    scores: np.ndarray | None
    times_ms: dict = field(default_factory=dict)
    pairs_total: int = 0
    pairs_unpruned: int = 0
    kernel_launches: int = 0
    t_pair_iter_ms: np.ndarray | None = None
    threshold_updates: int = 0
    waves: int = 0
    tile_pairs: int = 0
    empty_col_pairs: int = 0
    pad_row_pairs: int = 0


def _torch():
    import torch
    return torch


def alloc_workspace(nbytes: int, device=None):
    """Device workspace (uint8 tensor, 256-byte aligned by the caching allocator)."""
    torch = _torch()
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device or "cuda")


def _addr(a) -> int:
    """Address of a numpy array or torch tensor."""
    return a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr()


def _data_ptr(X):
    """(pointer, p, n, dtype, keepalive) of a numpy array or torch tensor."""
    if isinstance(X, np.ndarray):
        if X.dtype not in (np.float32, np.float64):
            X = X.astype(np.float64)
        X = np.ascontiguousarray(X)
        return X.ctypes.data, X.shape[0], X.shape[1], X.dtype, X
    torch = _torch()
    if isinstance(X, torch.Tensor):
        if X.dtype not in (torch.float32, torch.float64):
            X = X.double()
        X = X.contiguous()
        dt = np.float32 if X.dtype == torch.float32 else np.float64
        return X.data_ptr(), X.shape[0], X.shape[1], dt, X
    raise TypeError("X must be a numpy array or a torch tensor (p x n)")


def fit(X, precision: str = "mixed", prune: bool = True, reuse: bool = True, forced_order=None,
        want_scores: bool = False, want_B: bool = True, split_n: int = 0, timeout_s: float = 10.0,
        stream=None, workspace=None, max_iters: int = 0, timing: bool = False, out=None,
        tile_i: int = 0, tile_j: int = 0, prior=None, gamma0: float = 0.0, gamma_c: float = 2.0) -> FitResult:
    """lingam_fit on X (p x n, numpy on the host or a torch tensor on the GPU).  prior: None
    or a p x p int8 array, prior[i, j] = 1 when X_j is a known ancestor of X_i.  gamma0 > 0:
    the paper's threshold schedule (start gamma0, growth gamma_c) instead of the running bound."""
    L = load()
    ptr, p, n, dt, keep = _data_ptr(X)
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    o, keep_forced = make_opts(precision, dt, prune, reuse, split_n, timeout_s, stream, forced_order, max_iters,
                               timing, tile_i, tile_j, prior, gamma0, gamma_c)
    need = int(L.lingam_workspace_size(p, n, ctypes.byref(o)))
    if need == 0:
        raise LingamError(LINGAM_EINVAL, "invalid sizes or options")
    if workspace is None or workspace.numel() < need:
        workspace = alloc_workspace(need)
    if out is not None:            # caller-provided (e.g. pinned) host buffers for order and B
        order, B = out
    else:
        order = np.zeros(p, dtype=np.int32)
        B = np.zeros((p, p)) if want_B else None
    rs = np.zeros(p)
    mg = np.zeros(p)
    pe = np.zeros(p, dtype=np.int64)
    sc = np.full((p, p), np.nan) if want_scores else None
    rep = Report()
    rep.root_score = rs.ctypes.data_as(_c_dbl_p)
    rep.margin_lb = mg.ctypes.data_as(_c_dbl_p)
    rep.pairs_evaluated = pe.ctypes.data_as(_c_ll_p)
    if sc is not None:
        rep.scores = sc.ctypes.data_as(_c_dbl_p)
    tpi = np.zeros(p) if timing else None
    if tpi is not None:
        rep.t_pair_iter_ms = tpi.ctypes.data_as(_c_dbl_p)
    st = L.lingam_fit(ctypes.c_void_p(ptr), p, n, _addr(order), _addr(B) if B is not None else None,
                      ctypes.c_void_p(workspace.data_ptr()), ctypes.byref(o), ctypes.byref(rep))
    del keep, keep_forced
    if st != LINGAM_OK:
        raise LingamError(st, status_string(st))
    return FitResult(order=order, B=B, root_score=rs, margin_lb=mg, pairs_evaluated=pe, scores=sc,
                     times_ms={"standardize": rep.t_standardize_ms, "gram": rep.t_gram_ms,
                               "order": rep.t_order_ms, "B": rep.t_B_ms, "pair": rep.t_pair_ms,
                               "compute": rep.t_compute_ms, "merge": rep.t_merge_ms, "remove": rep.t_remove_ms},
                     pairs_total=int(rep.pairs_total), pairs_unpruned=int(rep.pairs_unpruned),
                     kernel_launches=int(rep.kernel_launches), t_pair_iter_ms=tpi,
                     threshold_updates=int(rep.threshold_updates), waves=int(rep.waves),
                     tile_pairs=int(rep.tile_pairs), empty_col_pairs=int(rep.empty_col_pairs),
                     pad_row_pairs=int(rep.pad_row_pairs))


def covariance(X, precision: str = "mixed", stream=None, workspace=None, out=None):
    """lingam_covariance: Sigma (p x p, float64) of the normalised rows of X, and the
    report's {"standardize", "gram"} times in ms.  `out` may be a float64 numpy array
    or a CUDA tensor (p x p) to write Sigma into."""
    L = load()
    ptr, p, n, dt, keep = _data_ptr(X)
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    o, _ = make_opts(precision, dt, stream=stream)
    need = int(L.lingam_workspace_size(p, n, ctypes.byref(o)))
    if need == 0:
        raise LingamError(LINGAM_EINVAL, "invalid sizes or options")
    if workspace is None or workspace.numel() < need:
        workspace = alloc_workspace(need)
    S = out if out is not None else np.zeros((p, p))
    rep = Report()
    st = L.lingam_covariance(ctypes.c_void_p(ptr), p, n, ctypes.c_void_p(_addr(S)),
                             ctypes.c_void_p(workspace.data_ptr()), ctypes.byref(o), ctypes.byref(rep))
    del keep
    if st != LINGAM_OK:
        raise LingamError(st, status_string(st))
    return S, {"standardize": rep.t_standardize_ms, "gram": rep.t_gram_ms,
               "kernel_launches": int(rep.kernel_launches)}


def tile_rows(p: int, n: int) -> int:
    """Tile rows the mixed path uses for a p x n problem (the autotuner's table)."""
    return int(load().lingam_tile_rows(p, n))


def tile_shape(p: int, n: int) -> tuple[int, int]:
    """(rows, columns) of the pair tiles the mixed path uses for a p x n problem."""
    L = load()
    return int(L.lingam_tile_rows(p, n)), int(L.lingam_tile_cols(p, n))


def autotune(X, stream=None, workspace=None):
    """lingam_autotune on X: times the ordering with 64x32, 32x32 and 64x16 pair tiles,
    records the fastest for X's size bucket; returns ((rows, cols), {shape: ms})."""
    L = load()
    ptr, p, n, dt, keep = _data_ptr(X)
    if stream is None:
        stream = _torch().cuda.current_stream().cuda_stream
    o, _ = make_opts("mixed", dt, stream=stream)
    need = int(L.lingam_workspace_size(p, n, ctypes.byref(o)))
    if workspace is None or workspace.numel() < need:
        workspace = alloc_workspace(need)
    tr, tc = ctypes.c_int(0), ctypes.c_int(0)
    ms = (ctypes.c_double * 3)()
    st = L.lingam_autotune(ctypes.c_void_p(ptr), p, n, ctypes.c_void_p(workspace.data_ptr()), ctypes.byref(o),
                           ctypes.byref(tr), ctypes.byref(tc), ms)
    del keep
    if st != LINGAM_OK:
        raise LingamError(st, status_string(st))
    return (int(tr.value), int(tc.value)), {(64, 32): float(ms[0]), (32, 32): float(ms[1]), (64, 16): float(ms[2])}


def autotune_batch(Xs, stream=None, workspace=None):
    """lingam_autotune_batch on a list of datasets: times lingam_fit_batch with 64x32, 32x32,
    64x16 and 32x16 pair tiles and the pair-per-warp mode (1x1), records the fastest for the
    bucket of the largest p and n;
    returns ((rows, cols), {shape: ms})."""
    L = load()
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    items = [_data_ptr(X) for X in Xs]
    count = len(items)
    o, _ = make_opts("mixed", items[0][3], stream=stream)
    pa = (ctypes.c_longlong * count)(*[it[1] for it in items])
    na = (ctypes.c_longlong * count)(*[it[2] for it in items])
    need = int(L.lingam_workspace_size_batch(count, pa, na, ctypes.byref(o)))
    if workspace is None or workspace.numel() < need:
        workspace = alloc_workspace(need)
    xp = (ctypes.c_void_p * count)(*[it[0] for it in items])
    tr, tc = ctypes.c_int(0), ctypes.c_int(0)
    ms = (ctypes.c_double * 5)()
    st = L.lingam_autotune_batch(count, xp, pa, na, ctypes.c_void_p(workspace.data_ptr()), ctypes.byref(o),
                                 ctypes.byref(tr), ctypes.byref(tc), ms)
    del items
    if st != LINGAM_OK:
        raise LingamError(st, status_string(st))
    return (int(tr.value), int(tc.value)), {(64, 32): float(ms[0]), (32, 32): float(ms[1]), (64, 16): float(ms[2]),
                                            (32, 16): float(ms[3]), (1, 1): float(ms[4])}


def batch_tile_shape(maxp: int, maxn: int) -> tuple[int, int]:
    """The pair-tile shape batch calls use for a batch whose largest problem is maxp x maxn."""
    L = load()
    return int(L.lingam_batch_tile_rows(maxp, maxn)), int(L.lingam_batch_tile_cols(maxp, maxn))


def autotune_reset():
    load().lingam_autotune_reset()


def selftest_wait(which: int, timeout_s: float) -> int:
    """lingam_selftest_wait: the status one device-side wait recorded after waiting for an
    event that never happens (0: mbarrier phase, 1: grid barrier, 2: wave word, 3: the B
    fit's Cholesky row flag)."""
    obs = ctypes.c_int(0)
    st = load().lingam_selftest_wait(int(which), float(timeout_s), ctypes.byref(obs))
    if st != LINGAM_OK:
        raise LingamError(st, status_string(st))
    return int(obs.value)


def _reports(count, ps, want_report, want_scores=False):
    """Report structs with host arrays for root scores, margins and pair counts (and the
    p x p per-iteration score matrices when want_scores is set)."""
    if not (want_report or want_scores):
        return None, None
    reps = (Report * count)()
    keep = []
    for k in range(count):
        rs, mg, pe = np.zeros(ps[k]), np.zeros(ps[k]), np.zeros(ps[k], dtype=np.int64)
        sc = np.full((ps[k], ps[k]), np.nan) if want_scores else None
        reps[k].root_score = rs.ctypes.data_as(_c_dbl_p)
        reps[k].margin_lb = mg.ctypes.data_as(_c_dbl_p)
        reps[k].pairs_evaluated = pe.ctypes.data_as(_c_ll_p)
        if sc is not None:
            reps[k].scores = sc.ctypes.data_as(_c_dbl_p)
        keep.append((rs, mg, pe, sc))
    return reps, keep


@dataclass
class BatchResult:
    status: int                    # first non-OK dataset status, else LINGAM_OK
    statuses: np.ndarray           # per dataset
    orders: list                   # per dataset, int32 [p]
    Bs: list | None                # per dataset, float64 [p, p]
    root_scores: list | None = None
    margins: list | None = None
    pairs: list | None = None
    scores: list | None = None     # per dataset, p x p (want_scores): S_v at iteration k, NaN if not complete


def batch_workspace(ps, ns, precision: str = "mixed", input_dtype=np.float32):
    """A device workspace for lingam_fit_batch over datasets of sizes ps[k] x ns[k];
    pass it to every call on these shapes to let the library replay its CUDA graph."""
    L = load()
    o, _ = make_opts(precision, input_dtype)
    count = len(ps)
    pa = (ctypes.c_longlong * count)(*ps)
    na = (ctypes.c_longlong * count)(*ns)
    need = int(L.lingam_workspace_size_batch(count, pa, na, ctypes.byref(o)))
    if need == 0:
        raise LingamError(LINGAM_EINVAL, "invalid sizes or options")
    return alloc_workspace(need)


def fit_batch(Xs, precision: str = "mixed", prune: bool = True, want_B: bool = True, stream=None, workspace=None,
              want_report: bool = False, want_scores: bool = False, tile_i: int = 0, tile_j: int = 0) -> BatchResult:
    """lingam_fit_batch over a list of datasets (numpy or torch, each p_k x n_k, one dtype);
    tile_i x tile_j: the pair-tile shape of the mixed path (0, 0: the batch autotuner's)."""
    L = load()
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    items = [_data_ptr(X) for X in Xs]
    count = len(items)
    if len({it[3] for it in items}) > 1:
        raise TypeError("all datasets of a batch must share one dtype")
    o, _ = make_opts(precision, items[0][3] if items else np.float32, prune, True, 0, 10.0, stream,
                     tile_i=tile_i, tile_j=tile_j)
    ps = [it[1] for it in items]
    ns = [it[2] for it in items]
    pa = (ctypes.c_longlong * count)(*ps)
    na = (ctypes.c_longlong * count)(*ns)
    need = int(L.lingam_workspace_size_batch(count, pa, na, ctypes.byref(o)))
    if need == 0:
        raise LingamError(LINGAM_EINVAL, "invalid sizes or options")
    if workspace is None or workspace.numel() < need:
        workspace = alloc_workspace(need)
    orders = [np.zeros(p, dtype=np.int32) for p in ps]
    Bs = [np.zeros((p, p)) for p in ps] if want_B else None
    xp = (ctypes.c_void_p * count)(*[it[0] for it in items])
    op = (ctypes.c_void_p * count)(*[o_.ctypes.data for o_ in orders])
    bp = (ctypes.c_void_p * count)(*[b.ctypes.data for b in Bs]) if Bs is not None else None
    status = np.zeros(count, dtype=np.int32)
    reps, keep_rep = _reports(count, ps, want_report, want_scores)
    st = L.lingam_fit_batch(count, xp, pa, na, op, bp, ctypes.c_void_p(workspace.data_ptr()), ctypes.byref(o),
                            status.ctypes.data_as(_c_int_p), reps)
    del items
    res = BatchResult(status=int(st), statuses=status, orders=orders, Bs=Bs)
    if keep_rep:
        res.root_scores = [k[0] for k in keep_rep]
        res.margins = [k[1] for k in keep_rep]
        res.pairs = [k[2] for k in keep_rep]
        if want_scores:
            res.scores = [k[3] for k in keep_rep]
    return res


def fit_bootstrap(X, idx, precision: str = "mixed", prune: bool = True, want_B: bool = True, stream=None,
                  workspace=None, want_report: bool = False, want_scores: bool = False, tile_i: int = 0,
                  tile_j: int = 0) -> BatchResult:
    """lingam_fit_bootstrap: X (p x n), idx (nboot x n column indices, numpy or CUDA tensor);
    tile_i x tile_j as for fit_batch."""
    L = load()
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    ptr, p, n, dt, keep = _data_ptr(X)
    if isinstance(idx, np.ndarray):
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        iptr, nboot = idx.ctypes.data, idx.shape[0]
    else:
        idx = idx.to(torch.int32).contiguous()
        iptr, nboot = idx.data_ptr(), idx.shape[0]
    if idx.shape[1] != n:
        raise ValueError("idx must be nboot x n")
    o, _ = make_opts(precision, dt, prune, True, 0, 10.0, stream, tile_i=tile_i, tile_j=tile_j)
    need = int(L.lingam_workspace_size_bootstrap(p, n, nboot, ctypes.byref(o)))
    if need == 0:
        raise LingamError(LINGAM_EINVAL, "invalid sizes or options")
    if workspace is None or workspace.numel() < need:
        workspace = alloc_workspace(need)
    order = np.zeros((nboot, p), dtype=np.int32)
    B = np.zeros((nboot, p, p)) if want_B else None
    status = np.zeros(nboot, dtype=np.int32)
    reps, keep_rep = _reports(nboot, [p] * nboot, want_report, want_scores)
    st = L.lingam_fit_bootstrap(ctypes.c_void_p(ptr), p, n, nboot, ctypes.c_void_p(iptr), order.ctypes.data,
                                B.ctypes.data if B is not None else None, ctypes.c_void_p(workspace.data_ptr()),
                                ctypes.byref(o), status.ctypes.data_as(_c_int_p), reps)
    del keep
    res = BatchResult(status=int(st), statuses=status, orders=list(order), Bs=list(B) if B is not None else None)
    if keep_rep:
        res.root_scores = [k[0] for k in keep_rep]
        res.margins = [k[1] for k in keep_rep]
        res.pairs = [k[2] for k in keep_rep]
        if want_scores:
            res.scores = [k[3] for k in keep_rep]
    return res


STATIC_SCRATCH_BYTES = 32 << 20   # LINGAM_STATIC_SCRATCH_BYTES in include/lingam.h


def fit_static(X, precision: str = "mixed", prune: bool = True, want_B: bool = True, want_scores: bool = False,
               stream=None) -> FitResult:
    """lingam_fit_static: the same fit as `fit`, run in the library's own
    fixed scratch area instead of a caller-provided workspace, for callers
    that cannot allocate device memory.  Raises LingamError(EINVAL) when the
    problem's workspace would exceed STATIC_SCRATCH_BYTES."""
    L = load()
    ptr, p, n, dt, keep = _data_ptr(X)
    if stream is None:
        stream = _torch().cuda.current_stream().cuda_stream
    o, _ = make_opts(precision, dt, prune, True, 0, 10.0, stream)
    order = np.zeros(p, dtype=np.int32)
    B = np.zeros((p, p)) if want_B else None
    rs, mg, pe = np.zeros(p), np.zeros(p), np.zeros(p, dtype=np.int64)
    sc = np.full((p, p), np.nan) if want_scores else None
    rep = Report()
    rep.root_score = rs.ctypes.data_as(_c_dbl_p)
    rep.margin_lb = mg.ctypes.data_as(_c_dbl_p)
    rep.pairs_evaluated = pe.ctypes.data_as(_c_ll_p)
    if sc is not None:
        rep.scores = sc.ctypes.data_as(_c_dbl_p)
    st = L.lingam_fit_static(ctypes.c_void_p(ptr), p, n, order.ctypes.data, B.ctypes.data if B is not None else None,
                             ctypes.byref(o), ctypes.byref(rep))
    del keep
    if st != LINGAM_OK:
        need = int(L.lingam_workspace_size(p, n, ctypes.byref(o)))
        msg = status_string(st)
        if st == LINGAM_EINVAL and need > STATIC_SCRATCH_BYTES:
            msg = f"problem needs {need} bytes of scratch, the static area holds {STATIC_SCRATCH_BYTES}"
        raise LingamError(st, msg)
    return FitResult(order=order, B=B, root_score=rs, margin_lb=mg, pairs_evaluated=pe, scores=sc,
                     times_ms={"standardize": rep.t_standardize_ms, "gram": rep.t_gram_ms,
                               "order": rep.t_order_ms, "B": rep.t_B_ms, "pair": rep.t_pair_ms},
                     pairs_total=int(rep.pairs_total), pairs_unpruned=int(rep.pairs_unpruned),
                     kernel_launches=int(rep.kernel_launches))

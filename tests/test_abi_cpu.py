"""CPU checks of the C ABI library: it builds, loads, and exports every
function include/lingam.h declares; the calls that need no GPU behave."""
import ctypes
import os

import numpy as np
import pytest

from paper_2109_13993_gb300 import build, lingam


@pytest.fixture(scope="module")
def lib():
    build.build()
    return lingam.load()


def test_exports_every_declared_symbol(lib):
    names = lingam.header_functions()
    assert {"lingam_fit", "lingam_fit_batch", "lingam_workspace_size", "lingam_status_string",
            "lingam_default_opts", "lingam_workspace_size_batch"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name


def test_default_opts(lib):
    o = lingam.Opts()
    lib.lingam_default_opts(ctypes.byref(o))
    assert o.precision == lingam.LINGAM_MIXED and o.input_dtype == lingam.LINGAM_F32
    assert o.prune == 1 and o.reuse == 1 and o.timeout_s == 10.0 and not o.stream and not o.forced_order


def test_status_strings(lib):
    for s in (0, -1, -2, -3, -4, -5):
        assert lingam.status_string(s)
    assert lingam.status_string(0) == "ok"
    assert lingam.status_string(123) == "unknown status"


def test_workspace_size(lib):
    a = lingam.workspace_size(100, 10000)
    b = lingam.workspace_size(1000, 10000)
    c = lingam.workspace_size(1000, 10000, precision="fp64")
    assert 0 < a < b and a < c   # the mixed path also holds the Gram's digit planes
    assert b % 256 == 0
    assert lingam.workspace_size(0, 100) == 0
    assert lingam.workspace_size(10, 2) == 0
    o, _ = lingam.make_opts()
    o.precision = 7
    assert lib.lingam_workspace_size(10, 100, ctypes.byref(o)) == 0
    ps = (ctypes.c_longlong * 2)(10, 20)
    ns = (ctypes.c_longlong * 2)(100, 200)
    tot = lib.lingam_workspace_size_batch(2, ps, ns, None)
    assert tot >= lingam.workspace_size(10, 100) + lingam.workspace_size(20, 200)


def test_fit_rejects_bad_arguments_without_gpu_work(lib):
    # NULL pointers and bad sizes are rejected before any CUDA call
    assert lib.lingam_fit(None, 10, 100, None, None, None, None, None) == lingam.LINGAM_EINVAL
    x = np.zeros((3, 10), dtype=np.float32)
    order = np.zeros(3, dtype=np.int32)
    assert lib.lingam_fit(ctypes.c_void_p(x.ctypes.data), 3, 2, order.ctypes.data, None, None, None,
                          None) == lingam.LINGAM_EINVAL


def test_tile_rows_default_rule(lib):
    # the autotuner's default before any measurement: 64-row tiles
    lingam.autotune_reset()
    assert lingam.tile_rows(20, 2000) == 64
    assert lingam.tile_rows(1000, 10000) == 64
    assert lingam.tile_rows(0, 100) == 0
    assert lingam.tile_shape(1000, 10000) == (64, 32)
    # batches: a table of their own, untuned default the pair mode up to 128 variables
    assert lingam.batch_tile_shape(50, 2000) == (1, 1)
    assert lingam.batch_tile_shape(128, 8000) == (1, 1)
    assert lingam.batch_tile_shape(129, 2000) == (32, 32)
    assert lingam.batch_tile_shape(1000, 10000) == (32, 32)
    assert lib.lingam_batch_tile_rows(0, 100) == 0
    o, _ = lingam.make_opts()
    for ti, tj in ((16, 0), (48, 0), (128, 0), (0, 8), (0, 64), (32, 16)):
        o.tile_i, o.tile_j = ti, tj
        assert lib.lingam_workspace_size(10, 100, ctypes.byref(o)) == 0
    for ti, tj in ((64, 32), (32, 32), (64, 16), (0, 16), (32, 0)):
        o.tile_i, o.tile_j = ti, tj
        assert lib.lingam_workspace_size(10, 100, ctypes.byref(o)) > 0
    # 32 x 16 tiles are a batch shape: batch sizing accepts them, single fits do not
    o.tile_i, o.tile_j = 32, 16
    ps = (ctypes.c_longlong * 1)(10)
    ns = (ctypes.c_longlong * 1)(100)
    assert lib.lingam_workspace_size_batch(1, ps, ns, ctypes.byref(o)) > 0
    assert lib.lingam_workspace_size(10, 100, ctypes.byref(o)) == 0
    o.tile_i, o.tile_j = 1, 1   # the batch pair-per-warp mode
    assert lib.lingam_workspace_size_batch(1, ps, ns, ctypes.byref(o)) > 0
    assert lib.lingam_workspace_size(10, 100, ctypes.byref(o)) == 0
    o.tile_i, o.tile_j = 1, 32
    assert lib.lingam_workspace_size_batch(1, ps, ns, ctypes.byref(o)) == 0


def test_batch_and_bootstrap_workspace_sizes(lib):
    ps = (ctypes.c_longlong * 3)(10, 20, 50)
    ns = (ctypes.c_longlong * 3)(100, 200, 2000)
    tot = lib.lingam_workspace_size_batch(3, ps, ns, None)
    assert tot >= sum(lingam.workspace_size(p, n) for p, n in zip(ps, ns))
    assert tot % 256 == 0
    bad = (ctypes.c_longlong * 3)(10, 0, 50)
    assert lib.lingam_workspace_size_batch(3, bad, ns, None) == 0
    o, _ = lingam.make_opts()
    b = lib.lingam_workspace_size_bootstrap(50, 2000, 256, ctypes.byref(o))
    # the resample regions plus the shared source (p n floats) and the indices (nboot n ints)
    assert b >= 256 * lingam.workspace_size(50, 2000) + 50 * 2000 * 4 + 256 * 2000 * 4
    assert lib.lingam_workspace_size_bootstrap(50, 2000, 0, ctypes.byref(o)) == 0


def test_batch_rejects_bad_arguments_without_gpu_work(lib):
    x = np.zeros((3, 10), dtype=np.float32)
    xp = (ctypes.c_void_p * 1)(x.ctypes.data)
    ps = (ctypes.c_longlong * 1)(3)
    ns = (ctypes.c_longlong * 1)(10)
    order = np.zeros(3, dtype=np.int32)
    op = (ctypes.c_void_p * 1)(order.ctypes.data)
    # no workspace, then a host "workspace": both rejected before any device work
    assert lib.lingam_fit_batch(1, xp, ps, ns, op, None, None, None, None, None) == lingam.LINGAM_EINVAL
    ws = np.zeros(1 << 20, dtype=np.uint8)
    st = np.zeros(1, dtype=np.int32)
    assert lib.lingam_fit_batch(1, xp, ps, ns, op, None, ctypes.c_void_p(ws.ctypes.data), None,
                                st.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), None) == lingam.LINGAM_EINVAL
    idx = np.full((2, 10), 11, dtype=np.int32)   # out of range
    o2 = np.zeros((2, 3), dtype=np.int32)
    assert lib.lingam_fit_bootstrap(ctypes.c_void_p(x.ctypes.data), 3, 10, 2, ctypes.c_void_p(idx.ctypes.data),
                                    ctypes.c_void_p(o2.ctypes.data), None, ctypes.c_void_p(ws.ctypes.data), None,
                                    None, None) == lingam.LINGAM_EINVAL


def test_selftest_wait_rejects_bad_arguments_without_gpu_work(lib):
    obs = ctypes.c_int(-7)
    assert lib.lingam_selftest_wait(4, 0.05, ctypes.byref(obs)) == lingam.LINGAM_EINVAL
    assert lib.lingam_selftest_wait(-1, 0.05, ctypes.byref(obs)) == lingam.LINGAM_EINVAL
    assert lib.lingam_selftest_wait(0, 0.0, ctypes.byref(obs)) == lingam.LINGAM_EINVAL
    assert lib.lingam_selftest_wait(0, 120.0, ctypes.byref(obs)) == lingam.LINGAM_EINVAL
    assert lib.lingam_selftest_wait(0, 0.05, None) == lingam.LINGAM_EINVAL
    assert obs.value == -7


# The largest problems lingam_fit_static accepts, as stated in include/lingam.h (default
# options; FP64 input on the FP64 path): (precision, n, largest p).
STATIC_LIMITS = [("mixed", 10000, 128), ("mixed", 5000, 217), ("mixed", 1000, 430),
                 ("fp64", 10000, 74), ("fp64", 5000, 136), ("fp64", 1000, 333)]


@pytest.mark.parametrize("precision,n,pmax", STATIC_LIMITS)
def test_static_scratch_limits_stated_in_the_header(lib, precision, n, pmax):
    dt = np.float32 if precision == "mixed" else np.float64
    assert 0 < lingam.workspace_size(pmax, n, precision, dt) <= lingam.STATIC_SCRATCH_BYTES
    assert lingam.workspace_size(pmax + 1, n, precision, dt) > lingam.STATIC_SCRATCH_BYTES
    hdr = open(os.path.join(build.INCLUDE, "lingam.h")).read()
    assert f"p = {pmax} at\n" in hdr or f"p = {pmax} at " in hdr.replace("\n *     ", " ")


def test_prior_knowledge_is_validated_without_gpu_work(lib):
    # a cycle among the known ancestors, or a value outside -1..1, is rejected before any
    # device work (the fit would otherwise fail on the host "workspace" with the same code,
    # so the check is that the status is EINVAL for a valid workspace-free call too)
    p, n = 6, 50
    x = np.zeros((p, n), dtype=np.float32)
    order = np.zeros(p, dtype=np.int32)
    for bad in ("cycle", "value"):
        prior = -np.ones((p, p), dtype=np.int8)
        if bad == "cycle":
            prior[1, 2] = prior[2, 4] = prior[4, 1] = 1
        else:
            prior[0, 3] = 5
        o, keep = lingam.make_opts(prior=prior)
        assert lib.lingam_fit(ctypes.c_void_p(x.ctypes.data), p, n, ctypes.c_void_p(order.ctypes.data), None,
                              None, ctypes.byref(o), None) == lingam.LINGAM_EINVAL
    # the workspace of a fit with prior knowledge holds the p x p matrix and the counts
    o, keep = lingam.make_opts(prior=-np.ones((p, p), dtype=np.int8))
    assert lib.lingam_workspace_size(100, 1000, ctypes.byref(o)) >= lingam.workspace_size(100, 1000) + 100 * 100


def test_threshold_schedule_options_are_validated(lib):
    """opts.gamma0 > 0 (the paper's threshold schedule) needs gamma_c > 1 and pruning with
    reuse; negative or non-finite values, and batches, are rejected without device work."""
    def size(**kw):
        o, _ = lingam.make_opts(**kw)
        return lib.lingam_workspace_size(50, 1000, ctypes.byref(o))
    assert size(gamma0=1e-3, gamma_c=2.0) == size() > 0
    for kw in ({"gamma0": -1.0}, {"gamma0": float("nan")}, {"gamma0": float("inf")},
               {"gamma0": 1e-3, "gamma_c": 1.0}, {"gamma0": 1e-3, "gamma_c": float("inf")},
               {"gamma0": 1e-3, "prune": False}, {"gamma0": 1e-3, "reuse": False}):
        assert size(**kw) == 0, kw
    o = lingam.Opts()
    lib.lingam_default_opts(ctypes.byref(o))
    assert o.gamma0 == 0.0 and o.gamma_c == 2.0
    x = np.zeros((3, 10), dtype=np.float32)
    xp = (ctypes.c_void_p * 1)(x.ctypes.data)
    ps = (ctypes.c_longlong * 1)(3)
    ns = (ctypes.c_longlong * 1)(10)
    order = np.zeros(3, dtype=np.int32)
    op = (ctypes.c_void_p * 1)(order.ctypes.data)
    ws = np.zeros(1 << 20, dtype=np.uint8)
    og, _ = lingam.make_opts(gamma0=1e-3)
    assert lib.lingam_fit_batch(1, xp, ps, ns, op, None, ctypes.c_void_p(ws.ctypes.data), ctypes.byref(og),
                                None, None) == lingam.LINGAM_EINVAL

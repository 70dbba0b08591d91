"""lingam_fit_static, the entry point for callers that cannot allocate
device memory (for instance a host program without a device allocator, or a
plug-in inside an application whose memory pool owns the GPU): it must give
the same result as lingam_fit, which takes a caller-provided workspace, on
two calls in a row (the second call finds the first call's leftovers in the
shared static scratch area).  Both run the same deterministic kernels on the
same inputs, so orders, B and scores must be bit-identical.  Also checked:
the largest problems the header states the static area admits run and match,
and the next size up is rejected.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle  # noqa: F401  (same import set as the other GPU tests)
from paper_2109_13993_gb300 import build, lingam, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lingam.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _same(got, ref):
    assert np.array_equal(got.order, ref.order)
    assert np.array_equal(got.B, ref.B)
    assert np.array_equal(np.isnan(got.scores), np.isnan(ref.scores))
    m = ~np.isnan(ref.scores)
    assert np.array_equal(got.scores[m], ref.scores[m])
    assert np.array_equal(got.root_score, ref.root_score)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_static_entry_point_matches_lingam_fit_twice(precision):
    dt = torch.float32 if precision == "mixed" else torch.float64
    for call, seed in enumerate((11, 12)):
        d = synth.lingam_dataset(45, 1700, 0.1, seed=seed)
        X = torch.tensor(d.X, dtype=dt, device="cuda")
        ref = lingam.fit(X, precision=precision, want_scores=True)
        got = lingam.fit_static(X, precision=precision, want_scores=True)
        _same(got, ref)


# the largest sizes include/lingam.h states for n = 10^4 (and the test of the statement
# against lingam_workspace_size runs on the CPU: tests/test_abi_cpu.py)
@pytest.mark.parametrize("precision,pmax", [("mixed", 128), ("fp64", 74)])
def test_static_entry_point_at_its_stated_limit(precision, pmax):
    n = 10000
    dt = torch.float32 if precision == "mixed" else torch.float64
    d = synth.lingam_dataset(pmax, n, 4.0 / (pmax - 1), seed=31)
    X = torch.tensor(d.X, dtype=dt, device="cuda")
    ref = lingam.fit(X, precision=precision, want_scores=True)
    got = lingam.fit_static(X, precision=precision, want_scores=True)
    _same(got, ref)
    d1 = synth.lingam_dataset(pmax + 1, n, 4.0 / pmax, seed=32)
    with pytest.raises(lingam.LingamError) as e:
        lingam.fit_static(torch.tensor(d1.X, dtype=dt, device="cuda"), precision=precision)
    assert e.value.status == lingam.LINGAM_EINVAL and "static area" in str(e.value)


def test_static_entry_point_rejects_too_large_problems():
    L = lingam.load()
    o, _ = lingam.make_opts("mixed", np.float32)
    p, n = 400, 20000
    assert L.lingam_workspace_size(p, n, ctypes.byref(o)) > lingam.STATIC_SCRATCH_BYTES
    X = torch.zeros((p, n), dtype=torch.float32, device="cuda")
    with pytest.raises(lingam.LingamError) as e:
        lingam.fit_static(X)
    assert e.value.status == lingam.LINGAM_EINVAL and "static area" in str(e.value)

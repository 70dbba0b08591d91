"""Failure detection on the GPU without a GPU fault: each kind of device-side wait of the
library (copy-ring mbarrier and grid barrier of the iteration and batch kernels, wave
word, the B fit's Cholesky row flag) is made to wait for an event that never happens; it
must give up after the timeout, record LINGAM_ETIMEOUT, and let the kernel end, so that
the context stays usable (a fit and a batch right after it succeed)."""
import time

import numpy as np
import pytest

from paper_2109_13993_gb300 import lingam, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2109_13993_gb300 import build
    build.build()
    lingam.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


@pytest.mark.parametrize("which", [0, 1, 2, 3])
def test_wait_gives_up_with_timeout_status(which):
    t0 = time.perf_counter()
    status = lingam.selftest_wait(which, 0.05)
    dt = time.perf_counter() - t0
    assert status == lingam.LINGAM_ETIMEOUT
    assert dt >= 0.05
    assert dt < 30.0
    # the context is still usable
    d = synth.lingam_dataset(8, 600, 0.4, seed=11)
    X = torch.tensor(d.X.astype(np.float32), device="cuda")
    r = lingam.fit(X, precision="mixed")
    assert sorted(r.order.tolist()) == list(range(8))
    rb = lingam.fit_batch([X, X[:5]], precision="mixed")
    assert rb.status == 0 and sorted(rb.orders[0].tolist()) == list(range(8))


@pytest.mark.parametrize("step", ["standardize", "covariance", "iteration:3", "bfit", "batch"])
def test_injected_host_fault_is_reported_and_the_next_call_succeeds(step, monkeypatch):
    """LINGAM_FAULT makes one step of a call report a failed launch on the host (no GPU
    fault): the call returns LINGAM_ECUDA, writes no output, and the next call succeeds."""
    d = synth.lingam_dataset(10, 800, 0.4, seed=12)
    X = torch.tensor(d.X.astype(np.float32), device="cuda")
    ref = lingam.fit(X, precision="mixed")
    monkeypatch.setenv("LINGAM_FAULT", step)
    if step == "batch":
        r = lingam.fit_batch([X, X[:6]], precision="mixed")
        assert r.status == lingam.LINGAM_ECUDA
    else:
        with pytest.raises(lingam.LingamError) as e:
            lingam.fit(X, precision="mixed")
        assert e.value.status == lingam.LINGAM_ECUDA
    monkeypatch.delenv("LINGAM_FAULT")
    again = lingam.fit(X, precision="mixed")
    assert np.array_equal(again.order, ref.order) and np.array_equal(again.B, ref.B)


def test_call_log_on_stderr():
    """LINGAM_LOG=1: one line per call on stderr with the sizes and the status."""
    import subprocess
    import sys
    code = ("import numpy as np, torch; from paper_2109_13993_gb300 import lingam, synth; "
            "d = synth.lingam_dataset(7, 500, 0.4, seed=3); "
            "lingam.fit(torch.tensor(d.X.astype(np.float32), device='cuda'))")
    env = dict(__import__("os").environ, LINGAM_LOG="1")
    root = __import__("os").path.dirname(__import__("os").path.dirname(__import__("os").path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert "lingam: fit p=7 n=500 precision=mixed status=0 (ok)" in r.stderr

"""Failure detection on the GPU without a GPU fault: each kind of device-side wait of
the iteration kernel (copy-ring mbarrier, grid barrier, wave word) is made to wait for
an event that never happens; it must give up after the timeout, record
LINGAM_ETIMEOUT, and let the kernel end, so that the context stays usable (a fit
right after it succeeds)."""
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


@pytest.mark.parametrize("which", [0, 1, 2])
def test_wait_gives_up_with_timeout_status(which):
    t0 = time.perf_counter()
    status = lingam.selftest_wait(which, 0.05)
    dt = time.perf_counter() - t0
    assert status == lingam.LINGAM_ETIMEOUT
    assert dt >= 0.05
    assert dt < 30.0
    # the context is still usable
    d = synth.lingam_dataset(8, 600, 0.4, seed=11)
    r = lingam.fit(torch.tensor(d.X.astype(np.float32), device="cuda"), precision="mixed")
    assert sorted(r.order.tolist()) == list(range(8))

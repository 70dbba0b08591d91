"""The debug build (every kernel's index bound checks compiled in, LINGAM_BOUNDS_CHECK): single
fits on both paths, a batch, bootstraps and the static entry point run through it without a
failed check (a failed check would return LINGAM_EBOUNDS), and give the release build's
results bit for bit (the checks guard accesses, they change no arithmetic)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2109_13993_gb300 import build, lingam, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RUN = r'''
import json, numpy as np, torch
from paper_2109_13993_gb300 import lingam, synth
out = {}
d = synth.lingam_dataset(70, 1500, 0.06, seed=41)
X32 = torch.tensor(d.X.astype(np.float32), device="cuda")
X64 = torch.tensor(d.X, device="cuda")
r = lingam.fit(X32, want_scores=True); out["mixed"] = [r.order.tolist(), r.B.ravel().tolist()]
r = lingam.fit(X64, precision="fp64"); out["fp64"] = [r.order.tolist(), r.B.ravel().tolist()]
r = lingam.fit(X32, tile_i=32, tile_j=32); out["mixed32"] = [r.order.tolist(), r.B.ravel().tolist()]
r = lingam.fit(X32, tile_i=64, tile_j=16); out["mixed16"] = [r.order.tolist(), r.B.ravel().tolist()]
ds = synth.uneven_batch(5, seed=3)
rb = lingam.fit_batch([torch.tensor(x.X[:, :1200].astype(np.float32), device="cuda") for x in ds])
out["batch"] = [int(rb.status), [o.tolist() for o in rb.orders]]
idx = synth.bootstrap_indices(1500, 6, seed=2)
rs = lingam.fit_bootstrap(X32[:20], idx)
out["boot"] = [int(rs.status), [o.tolist() for o in rs.orders]]
r = lingam.fit_static(X32); out["static"] = [r.order.tolist(), r.B.ravel().tolist()]
print("RESULT" + json.dumps(out))
'''


def _run(lib):
    env = dict(os.environ, LINGAM_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", RUN], env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT")][-1]
    return json.loads(line[len("RESULT"):])


def test_debug_build_runs_clean_and_matches_release():
    rel = _run(build.build())
    dbg = _run(build.build(debug=True))
    assert dbg["batch"][0] == 0 and dbg["boot"][0] == 0
    for key in rel:
        assert dbg[key] == rel[key], key

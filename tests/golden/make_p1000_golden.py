"""Writes p1000_n10000_seed1_iters0_4.txt: the FP64 oracle's complete scores at the first
five iterations of DirectLiNGAM (Algorithm 1 with FindRoot of Algorithm 2) on the
p = 1000, n = 10^4 workload of the benchmark (seed 1, FP32-representable data).

Iteration k scores every variable left after the oracle's own first k roots: S_v of
Algorithm 2 (sum over all partners of min(0, I)^2, Eq. Itest with Eq. HApp), each root the
argmin (lowest index on ties).  Only oracle/ computes anything here; synth only draws the
seeded input.  Takes a few minutes on a multi-core host:

    python tests/golden/make_p1000_golden.py
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2109_13993_gb300 import synth  # noqa: E402

OUT = os.path.join(HERE, "p1000_n10000_seed1_iters0_4.txt")
ITERS = 5


def main() -> None:
    d = synth.workload("p1000_n10000", seed=1)
    X64 = d.X.astype(np.float32).astype(np.float64)
    p = X64.shape[0]
    prefix: list[int] = []
    lines = ["# Oracle (FP64 CPU DirectLiNGAM, Algorithms 1-2, Eqs. Itest and HApp) scores of the",
             "# p=1000, n=10000 workload, seed 1, data rounded to FP32 and promoted to FP64.",
             "# Written by tests/golden/make_p1000_golden.py (calls oracle/ only).",
             "# Block per iteration k: 'ITER k ROOT v MARGIN m', then one line 'v S_v' per remaining",
             "# variable in index order (the variables of the prefix are absent).",
             f"# host: {os.cpu_count()} cores"]
    for k in range(ITERS):
        alive = np.array([v for v in range(p) if v not in set(prefix)], dtype=np.int32)
        t0 = time.perf_counter()
        S = oracle.variable_scores(X64, np.array(prefix, dtype=np.int32), alive)
        dt = time.perf_counter() - t0
        o = np.lexsort((alive, S))
        root = int(alive[o[0]])
        margin = float(S[o[1]] - S[o[0]])
        lines.append(f"ITER {k} ROOT {root} MARGIN {margin:.17g}")
        lines.extend(f"{int(v)} {float(s):.17g}" for v, s in zip(alive, S))
        prefix.append(root)
        print(f"iteration {k}: root {root}, margin {margin:.3e}, {dt:.1f} s", flush=True)
    with open(OUT, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()

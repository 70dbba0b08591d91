#!/usr/bin/env python
"""Benchmark of the DirectLiNGAM causal-ordering hot path on GB300.

Workload: seeded synthetic LiNGAM data, p = 1000 variables, n = 10^4 samples,
expected in-degree 2, FP32 storage (40 MB); mixed-precision path with
threshold pruning and pair reuse.  One step = one full lingam_fit call
(normalise, covariance, all p iterations of ordering, B fit) on inputs already
resident in HBM.  Metric: pair-sample evaluations per second, counted as the
unpruned-equivalent work sum_r r(r-1)/2 * n of one ordering (higher is better).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank fits its own dataset (seed = rank + 1): independent
problems, weak scaling, no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

P_DEFAULT, N_DEFAULT = 1000, 10000
# One metric and workload description for both arms (the reference arm is the FP64 CPU
# oracle on the same data).
METRIC = "pair-sample evals/s (unpruned-equivalent) at p=1000, n=1e4"


def workload_name(p: int, n: int) -> str:
    return f"p{p}_n{n} LiNGAM, expected in-degree 2, FP32-representable data, seed = rank+1"


L2_FLUSH_BYTES = 256 << 20
# Pair kernel SFU roofline: per pair-sample 4 ex2 (32 per SM per clock on sm_103a)
# plus 2 lg2 per 32 samples (16 per SM per clock).
SFU_CLK_PER_PAIR_SAMPLE = 4.0 / 32.0 + (2.0 / 32.0) / 16.0
# DRAM bytes (read + write) per launch of the iteration kernel, from an ncu capture of
# the current kernel version (profiles/); None until the current version is captured.
ITER_TRAFFIC_BYTES = 71.6e6   # ncu dram__bytes_read.sum + dram__bytes_write.sum, iteration 2 (55.1 + 16.5 MB)


def unpruned_pair_samples(p: int, n: int) -> float:
    return float(sum(r * (r - 1) // 2 for r in range(2, p + 1))) * n


def dataset_seed(rank: int) -> int:
    """Every rank fits its own independent dataset (weak scaling)."""
    return 1 + rank


def shard(count: int, world: int, rank: int) -> list[int]:
    """Datasets of a batch owned by `rank`: a contiguous, balanced block."""
    lo = count * rank // world
    hi = count * (rank + 1) // world
    return list(range(lo, hi))


def max_over_ranks(value: float, dist, device) -> float:
    """Largest value over all ranks (the job takes as long as its slowest rank)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks() -> dict:
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ------------------------------------------------------------------ clocks during the timed region
class ClockSampler:
    FIELDS = ("pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = (bus_id or "").lower()
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            if self.bus_id and self.bus_id[-12:] not in parts[0].lower():
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5], parts[6], parts[7], parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        top = max(r[0] for r in rows)
        loaded = [r for r in rows if r[0] >= 0.5 * top] or rows
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[k] for r in loaded for k in range(4) if r[2 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ CPU oracle leg
def oracle_rate(X64: np.ndarray, target_s: float, seed: int = 7):
    """Oracle FindRoot (Algorithm 2) over a subset of m variables, m sized so the
    call takes about target_s seconds on all host cores.  Returns
    (pair-samples/s, seconds, m, threads) in unpruned-equivalent units."""
    import oracle
    n = X64.shape[1]
    rng = np.random.default_rng(seed)
    m0 = 24
    U0 = np.sort(rng.choice(X64.shape[0], m0, replace=False))
    t = time.perf_counter()
    oracle.find_root_scores(X64, U0)
    t0 = max(time.perf_counter() - t, 1e-3)
    m = int(min(X64.shape[0], max(m0, np.sqrt(target_s / t0 * m0 * (m0 - 1)))))
    U = np.sort(rng.choice(X64.shape[0], m, replace=False))
    t = time.perf_counter()
    oracle.find_root_scores(X64, U)
    dt = time.perf_counter() - t
    return m * (m - 1) / 2 * n / dt, dt, m, oracle.num_threads(0)


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    from paper_2109_13993_gb300 import synth
    d = synth.workload("p1000_n10000", seed=1)
    X64 = d.X.astype(np.float32).astype(np.float64)
    per_step_target = 8.0
    for _ in range(args.warmup):
        oracle_rate(X64, per_step_target)
    rates, times, ms = [], [], []
    for _ in range(args.steps):
        r, dt, m, cores = oracle_rate(X64, per_step_target)
        rates.append(r)
        times.append(dt)
        ms.append(m)
    value = float(np.mean(rates))
    sample = (f"oracle FindRoot (Algorithm 2, every ordered pair) over {int(np.mean(ms))} of the 1000 variables "
              f"of the p=1000, n=10000 dataset per step; rate in unpruned-equivalent pair-samples")
    line = {"impl": "reference", "metric": METRIC,
            "value": value, "unit": "pair-samples/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * float(np.mean(times)), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(P_DEFAULT, N_DEFAULT), "p": P_DEFAULT, "n": N_DEFAULT,
                       "arm": "FP64 CPU oracle, every ordered pair (no pruning)"},
            "cpu_baseline": {"value": value, "unit": "pair-samples/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "pair-samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU leg
def batched_workload(lingam, synth, torch, dev, stream, reps: int = 5) -> dict:
    """The batched configuration: 256 bootstrap resamples of one p=50, n=2000 dataset
    and 64 datasets with p in 20..120, n in 500..8000 (FP32, mixed path), each set one
    library call; inputs resident on the device; after two calls (eager, graph capture)
    the replayed graph is timed with CUDA events, with every tile shape of the batch kernel
    and with the shape the batch autotuner picks for each set.  Next to it, every member of
    each set as a sequential single fit through lingam_fit (one workspace reused), timed as
    a whole."""
    import ctypes
    d = synth.lingam_dataset(50, 2000, 4.0 / 49.0, seed=5)
    X = torch.tensor(d.X.astype(np.float32), device=dev)
    idx = torch.tensor(synth.bootstrap_indices(2000, 256, seed=6), device=dev)
    ds = synth.uneven_batch(64, seed=7)
    Xs = [torch.tensor(dd.X.astype(np.float32), device=dev) for dd in ds]
    o, _ = lingam.make_opts()
    wsb = lingam.alloc_workspace(lingam.load().lingam_workspace_size_bootstrap(50, 2000, 256, ctypes.byref(o)),
                                 device=dev)
    wsu = lingam.batch_workspace([x.shape[0] for x in Xs], [x.shape[1] for x in Xs])

    def timed(fn):
        out = []
        for _ in range(2):
            fn()
        for _ in range(reps):
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            assert r.status == 0
            out.append(e0.elapsed_time(e1))
        return float(np.median(out))

    # every tile shape of the batch kernel on both sets, then the batch autotuner's choice
    # for each set's size bucket (the gathered resamples stand in for the bootstrap call)
    Xb = [X[:, idx[b].long()].contiguous() for b in range(idx.shape[0])]
    shapes_ms = {"bootstrap_256": {}, "uneven_64": {}}
    for ti, tj in ((64, 32), (32, 32), (64, 16), (32, 16), (1, 1)):
        shapes_ms["bootstrap_256"][f"{ti}x{tj}"] = timed(
            lambda: lingam.fit_bootstrap(X, idx, workspace=wsb, tile_i=ti, tile_j=tj))
        shapes_ms["uneven_64"][f"{ti}x{tj}"] = timed(lambda: lingam.fit_batch(Xs, workspace=wsu, tile_i=ti, tile_j=tj))
    lingam.autotune_reset()
    tuned = {"bootstrap_256": lingam.autotune_batch(Xb)[0], "uneven_64": lingam.autotune_batch(Xs, workspace=wsu)[0]}
    t_boot = timed(lambda: lingam.fit_bootstrap(X, idx, workspace=wsb))
    t_unev = timed(lambda: lingam.fit_batch(Xs, workspace=wsu))
    # useful work: the pairs each problem's fit evaluated (reports of one more call) x its n
    rb = lingam.fit_bootstrap(X, idx, workspace=wsb, want_report=True)
    ru = lingam.fit_batch(Xs, workspace=wsu, want_report=True)
    ps_boot = sum(float(np.sum(pp)) * 2000 for pp in rb.pairs)
    ps_unev = sum(float(np.sum(pp)) * x.shape[1] for pp, x in zip(ru.pairs, Xs))
    # every member as a sequential single fit (one workspace of the largest size, reused)
    ws1 = lingam.alloc_workspace(lingam.workspace_size(50, 2000), device=dev)
    for x in Xb[:2]:
        lingam.fit(x, workspace=ws1)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for x in Xb:
        lingam.fit(x, workspace=ws1)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    seq_boot = e0.elapsed_time(e1)
    wsm = lingam.alloc_workspace(max(lingam.workspace_size(x.shape[0], x.shape[1]) for x in Xs), device=dev)
    lingam.fit(Xs[0], workspace=wsm)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for x in Xs:
        lingam.fit(x, workspace=wsm)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    seq_unev = e0.elapsed_time(e1)
    return {"workload": "256 bootstrap resamples of p=50, n=2000 + 64 datasets p in 20..120, n in 500..8000",
            "bootstrap_256_ms": t_boot, "uneven_64_ms": t_unev,
            "sequential_single_fits_ms": {"bootstrap_256": seq_boot, "uneven_64": seq_unev},
            "speedup_vs_sequential": {"bootstrap_256": seq_boot / t_boot, "uneven_64": seq_unev / t_unev},
            "pair_samples_evaluated": {"bootstrap_256": ps_boot, "uneven_64": ps_unev},
            "pair_samples_per_s": {"bootstrap_256": ps_boot / (t_boot / 1e3), "uneven_64": ps_unev / (t_unev / 1e3)},
            "tile_shape": {k: f"{v[0]}x{v[1]}" for k, v in tuned.items()},
            "tile_shapes_ms": shapes_ms,
            "timing": "median of 5 graph replays, CUDA events; inputs on the device; tile shape chosen by "
                      "lingam_autotune_batch for each set's size bucket"}


def cpu_model() -> str:
    """The host CPU's model name (lscpu), else /proc/cpuinfo's model name or Arm part number."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    arm_parts = {"0xd4f": "Neoverse-V2", "0xd40": "Neoverse-V1", "0xd0c": "Neoverse-N1"}
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                v = line.split(":", 1)[1].strip()
                return arm_parts.get(v, v)
    except OSError:
        pass
    return "unknown"


def configs_table(lingam, synth, torch, dev, stream, seeds=(1, 2, 3, 4, 5), reps: int = 3) -> dict:
    """The five benchmark configurations over dataset seeds 1-5: fit time (median of
    `reps`, CUDA events, inputs on the device), pairs evaluated, and for the single-dataset
    configurations the FP64 GPU path on the same data (config 5: its first 5 iterations
    against the mixed path's first 5) and whether the two paths' orders agree."""
    def timed(fn):
        fn()
        out = []
        for _ in range(reps):
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            out.append(e0.elapsed_time(e1))
        return float(np.median(out)), r

    table = {}
    for name, dt_in in (("p20_n2000", np.float64), ("p100_n10000", np.float32), ("p300_n5000", np.float32),
                        ("p1000_n10000", np.float32)):
        rows = []
        for seed in seeds:
            d = synth.workload(name, seed=seed)
            p, n = d.X.shape
            row = {"seed": seed}
            X64 = torch.tensor(d.X.astype(np.float32).astype(np.float64) if dt_in == np.float32 else d.X, device=dev)
            k = 5 if p >= 1000 else 0
            if dt_in == np.float32:
                X32 = torch.tensor(d.X.astype(np.float32), device=dev)
                ws = lingam.alloc_workspace(lingam.workspace_size(p, n), device=dev)
                row["mixed_ms"], rm = timed(lambda: lingam.fit(X32, workspace=ws))
                row["mixed_pairs"] = int(rm.pairs_total)
                if k:
                    row["mixed_first5_ms"], rm5 = timed(lambda: lingam.fit(X32, workspace=ws, max_iters=k))
            ws64 = lingam.alloc_workspace(lingam.workspace_size(p, n, "fp64", np.float64), device=dev)
            row["fp64_ms" if not k else "fp64_first5_ms"], r64 = timed(
                lambda: lingam.fit(X64, precision="fp64", workspace=ws64, max_iters=k))
            if dt_in == np.float32:
                om, o64 = (rm5 if k else rm).order[:k or p], r64.order[:k or p]
                row["orders_agree"] = bool(np.array_equal(om, o64))
                if not row["orders_agree"]:
                    # where the two paths first part: the FP64 path's full scores at that
                    # iteration (same history up to it) for the two roots picked
                    it = int(np.argmax(om != o64))
                    s64 = lingam.fit(X64, precision="fp64", workspace=ws64, prune=False, want_scores=True,
                                     max_iters=it + 1).scores[it]
                    a, b = s64[int(o64[it])], s64[int(om[it])]
                    # the mixed path's per-score error bound at this iteration (kappa = 1.6e-6 as
                    # measured against the oracle, m = partners per variable)
                    m = p - it - 1
                    tau = 1.6e-6 * np.sqrt(m * max(float(b), 0.0)) + m * 4e-12
                    row["first_divergence"] = {"iteration": it, "fp64_score_fp64_root": float(a),
                                               "fp64_score_mixed_root": float(b),
                                               "relative_gap": float((b - a) / abs(a)) if a else None,
                                               "gap_over_mixed_score_bound": float((b - a) / tau)}
            rows.append(row)
            del ws64
        table[name] = rows
    boot, unev = [], []
    for seed in seeds:
        d = synth.lingam_dataset(50, 2000, 4.0 / 49.0, seed=4 + seed)
        X = torch.tensor(d.X.astype(np.float32), device=dev)
        idx = torch.tensor(synth.bootstrap_indices(2000, 256, seed=5 + seed), device=dev)
        ws = lingam.alloc_workspace(lingam.load().lingam_workspace_size_bootstrap(
            50, 2000, 256, __import__("ctypes").byref(lingam.make_opts()[0])), device=dev)
        lingam.fit_bootstrap(X, idx, workspace=ws)
        boot.append(timed(lambda: lingam.fit_bootstrap(X, idx, workspace=ws))[0])
        ds = synth.uneven_batch(64, seed=6 + seed)
        Xs = [torch.tensor(dd.X.astype(np.float32), device=dev) for dd in ds]
        wsu = lingam.batch_workspace([x.shape[0] for x in Xs], [x.shape[1] for x in Xs])
        lingam.fit_batch(Xs, workspace=wsu)
        unev.append(timed(lambda: lingam.fit_batch(Xs, workspace=wsu))[0])
    table["batched"] = {"bootstrap_256_ms": boot, "uneven_64_ms": unev}
    return table


def scalability_sweep(lingam, synth, torch, dev, stream, reps: int = 3) -> list:
    """The paper's scalability experiment (Sec. V-D): sparse and dense synthetic graphs
    (synth.scalability_dataset) for p in {100, 200, 500, 1000} and n in {1024, 2048, 4096,
    8192}, seed 1, FP32 data, mixed path with pruning and reuse: full lingam_fit time
    (median of `reps` after one untimed call, CUDA events, inputs on the device) and the
    fraction of pairs the threshold saved."""
    rows = []
    for dense in (False, True):
        for p in (100, 200, 500, 1000):
            for n in (1024, 2048, 4096, 8192):
                d = synth.scalability_dataset(p, n, dense, seed=1)
                X = torch.tensor(d.X.astype(np.float32), device=dev)
                ws = lingam.alloc_workspace(lingam.workspace_size(p, n), device=dev)
                r = lingam.fit(X, workspace=ws)
                ts = []
                for _ in range(reps):
                    torch.cuda.synchronize(dev)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    lingam.fit(X, workspace=ws)
                    e1.record(stream)
                    torch.cuda.synchronize(dev)
                    ts.append(e0.elapsed_time(e1))
                rows.append({"graph": "dense" if dense else "sparse", "p": p, "n": n,
                             "fit_ms": float(np.median(ts)), "pairs_evaluated": int(r.pairs_total),
                             "pruned_fraction": 1.0 - r.pairs_total / r.pairs_unpruned})
                del ws, X
    return rows


def ablation(lingam, synth, torch, dev, stream, reps: int = 3) -> dict:
    """The paper's two schedule claims measured on this GPU (Sec. III-A messaging, Sec. III-B
    threshold): the p=300, n=5000 and p=1000, n=1e4 workloads (seed 1, mixed path) with the
    threshold and the pair reuse on (the default), the threshold off, and both off; and the
    sample-axis split (stream-K, the default) against one CTA per tile (split_n = 1), also on
    a long-sample dataset (p=100, n=1e5); and the paper's own threshold schedule (gamma0
    raised by factors c, Algorithms 6 and 9) in place of the running bound, with the number of
    raises (each a kernel launch and read-back in the paper's host loop).  Full lingam_fit time
    (median of `reps` after one untimed call) and pairs evaluated."""
    out = {}
    cases = [(name, synth.workload(name, seed=1)) for name in ("p300_n5000", "p1000_n10000")]
    cases.append(("p100_n100000", synth.lingam_dataset(100, 100000, 4.0 / 99.0, seed=1)))
    for name, d in cases:
        X = torch.tensor(d.X.astype(np.float32), device=dev)
        p, n = X.shape
        ws = lingam.alloc_workspace(lingam.workspace_size(p, n), device=dev)
        rows = {}
        legs = [("threshold+messaging", dict()), ("split_n=1 (one CTA per tile)", dict(split_n=1))]
        if name != "p100_n100000":
            legs += [("messaging only", dict(prune=False)), ("neither", dict(prune=False, reuse=False))]
            # the paper's schedule from a start below every root score of this fit, and from
            # the median root score
            r0 = lingam.fit(X, workspace=ws)
            rs = r0.root_score[r0.root_score > 0]
            lo, med = 1e-3 * float(rs.min()), float(np.median(rs))
            legs += [(f"paper threshold gamma0={g0:.3g} c={c:g}", dict(gamma0=g0, gamma_c=c))
                     for g0, c in ((lo, 2.0), (lo, 10.0), (med, 2.0))]
        for label, kw in legs:
            r = lingam.fit(X, workspace=ws, **kw)
            ts = []
            for _ in range(reps):
                torch.cuda.synchronize(dev)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                lingam.fit(X, workspace=ws, **kw)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                ts.append(e0.elapsed_time(e1))
            rows[label] = {"fit_ms": float(np.median(ts)), "pair_evaluations": int(r.pairs_total), "_order": r.order}
            if "gamma0" in kw:
                rows[label]["threshold_updates"] = int(r.threshold_updates)
        ref = rows["threshold+messaging"]["_order"]
        for label, _ in legs:
            rows[label]["order_equal_to_default"] = bool(np.array_equal(rows[label].pop("_order"), ref))
        a = rows["threshold+messaging"]
        rows["speedup_from_stream_k"] = rows["split_n=1 (one CTA per tile)"]["fit_ms"] / a["fit_ms"]
        if "neither" in rows:
            b, c = rows["messaging only"], rows["neither"]
            rows["comparisons_saved_by_threshold"] = 1.0 - a["pair_evaluations"] / b["pair_evaluations"]
            rows["speedup_from_threshold"] = b["fit_ms"] / a["fit_ms"]
            rows["speedup_from_messaging"] = c["fit_ms"] / b["fit_ms"]
        out[name] = rows
        del ws
    return out


def run_ours(args, rank: int, world: int):
    import torch
    import __graft_entry__ as entry
    from paper_2109_13993_gb300 import lingam, synth

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    entry.build()
    p, n = args.p, args.n
    seed = dataset_seed(rank)
    d = synth.workload("p1000_n10000", seed=seed) if (p, n) == (P_DEFAULT, N_DEFAULT) else \
        synth.lingam_dataset(p, n, 4.0 / max(p - 1, 1), seed=seed)
    X = torch.tensor(d.X.astype(np.float32), device=dev)
    ws = lingam.alloc_workspace(lingam.workspace_size(p, n), device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def step(inp, out=None, timing=False):
        return lingam.fit(inp, precision="mixed", workspace=ws, timing=timing, out=out, max_iters=args.max_iters,
                          want_B=args.max_iters == 0)

    for _ in range(args.warmup):
        flush.zero_()
        step(X)
    props = torch.cuda.get_device_properties(dev)
    bus = getattr(props, "pci_bus_id", None)
    bus_id = f"{bus:02x}:00" if isinstance(bus, int) else None
    # the timed steps run the library as shipped (no per-launch events, no phase timers)
    step_ms, pairs, launches = [], [], []
    with ClockSampler(bus_id) as clk:
        for _ in range(args.steps):
            flush.zero_()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = step(X)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            step_ms.append(e0.elapsed_time(e1))
            pairs.append(res.pairs_total)
            launches.append(res.kernel_launches)
    clocks = clk.summary()
    # a separate pass with the library's instrumentation on: the iteration kernel's launch
    # times (CUDA events on the launching stream, one after each launch) for the roofline,
    # and CTA 0's phase timers
    pair_ms, phases = [], []
    for _ in range(max(1, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize(dev)
        rt = step(X, timing=True)
        pair_ms.append(rt.times_ms["pair"])
        phases.append((rt.times_ms["compute"], rt.times_ms["merge"], rt.times_ms["remove"]))
    barrier()
    tot_ms = max_over_ranks(float(np.sum(step_ms)), dist, dev)
    ms_per_step = tot_ms / args.steps
    work = unpruned_pair_samples(p, n) if args.max_iters == 0 else \
        float(sum(r * (r - 1) // 2 for r in range(p - args.max_iters + 1, p + 1))) * n
    value = world * work / (ms_per_step / 1000.0)

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    Xh = torch.tensor(d.X.astype(np.float32)).pin_memory()
    order_h = torch.empty(p, dtype=torch.int32).pin_memory()
    B_h = torch.empty((p, p), dtype=torch.float64).pin_memory()
    e2e_ms = []
    for k in range(0 if args.no_e2e else args.warmup + args.steps):
        flush.zero_()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lingam.fit(Xh, precision="mixed", workspace=ws, out=(order_h, B_h))
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if k >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_tot = max_over_ranks(float(np.sum(e2e_ms)) if e2e_ms else float("nan"), dist, dev)
    e2e_value = world * work / (e2e_tot / args.steps / 1000.0)

    # pair-kernel roofline (SFU bound), from the timed steps
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    nsm = props.multi_processor_count
    peak = nsm * (1.0 / SFU_CLK_PER_PAIR_SAMPLE) * sm_max * 1e6
    achieved = float(np.mean(pairs)) * n / (float(np.mean(pair_ms)) / 1000.0)
    traffic = ITER_TRAFFIC_BYTES if (p, n) == (P_DEFAULT, N_DEFAULT) else None
    roofline = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gpair-samples/s",
                "frac": achieved / peak, "traffic": traffic,
                "traffic_basis": "ncu dram__bytes_read+write of one launch (iteration 2 of a fit, cold caches)",
                "kernel": "k_iteration<float>",
                "timing_basis": "separate instrumented pass (one CUDA event after each launch); the timed steps run "
                                "without instrumentation",
                "peak_basis": f"SFU: 4 ex2 + 1/16 lg2 per pair-sample, {nsm} SMs x 32 ex2/clk at sm_max {sm_max:.0f} MHz"}
    # the same work over the pair-compute phases of the waves alone (device timer; the rest
    # of each launch is merging, wave finalisation, removal and grid barriers)
    ph = np.mean(np.array(phases), axis=0)
    comp = float(np.mean(pairs)) * n / (float(np.mean([x[0] for x in phases])) / 1000.0)
    roofline["compute_phase"] = {"achieved": comp / 1e9, "frac": comp / peak,
                                 "ms_per_step": {"pair_compute": ph[0], "merge_finalize": ph[1], "removal": ph[2]}}
    # the pair tiles' own efficiency: useful pairs over the pairs the waves' tiles computed
    roofline["waves_per_step"] = int(rt.waves)
    roofline["tile_pairs_per_step"] = int(rt.tile_pairs)
    roofline["useful_fraction_of_tile_pairs"] = float(rt.pairs_total) / max(1, int(rt.tile_pairs))
    waste = max(1, int(rt.tile_pairs) - int(rt.pairs_total))
    roofline["tile_waste_shares"] = {"empty_columns": rt.empty_col_pairs / waste, "row_padding": rt.pad_row_pairs / waste,
                                     "column_block_duplicates": 1.0 - (rt.empty_col_pairs + rt.pad_row_pairs) / waste}

    line = {"metric": METRIC if (p, n) == (P_DEFAULT, N_DEFAULT) else
            f"pair-sample evals/s (unpruned-equivalent) at p={p}, n={n}",
            "value": value, "unit": "pair-samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": workload_name(p, n),
                       "p": p, "n": n, "precision": "mixed", "prune": True, "reuse": True,
                       "l2": "flushed between steps (256 MB write)", "parallelism": f"independent datasets x{world}"},
            "ordering_ms": ms_per_step, "pairs_evaluated_per_step": int(np.mean(pairs)),
            "pairs_unpruned_per_step": int(work // n), "pruned_fraction": 1.0 - float(np.mean(pairs)) / (work / n),
            "gpu_launches": int(np.sum(launches)), "clocks": clocks, "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": "pair-samples/s", "h2d_bytes_per_step": int(p * n * 4),
                    "d2h_bytes_per_step": int(p * 4 + p * p * 8)}}

    if world == 1 and not args.no_fp64:
        # FP64 GPU path vs mixed path on the same first iterations (same unpruned work)
        k = args.fp64_iters
        Xd = torch.tensor(d.X, device=dev)
        ws64 = lingam.alloc_workspace(lingam.workspace_size(p, n, precision="fp64", input_dtype=np.float64), device=dev)
        lingam.fit(X, precision="mixed", workspace=ws, max_iters=2)
        rm = lingam.fit(X, precision="mixed", workspace=ws, max_iters=k)
        r64 = lingam.fit(Xd, precision="fp64", workspace=ws64, max_iters=k)
        w_k = float(sum(r * (r - 1) // 2 for r in range(p - k + 1, p + 1))) * n
        line["fp64_path"] = {"iterations": k, "mixed_order_ms": rm.times_ms["order"],
                             "fp64_order_ms": r64.times_ms["order"],
                             "mixed_pair_samples_per_s": w_k / (rm.times_ms["order"] / 1000.0),
                             "fp64_pair_samples_per_s": w_k / (r64.times_ms["order"] / 1000.0),
                             "mixed_speedup": r64.times_ms["order"] / rm.times_ms["order"],
                             "same_roots": bool(np.array_equal(rm.order[:k], r64.order[:k]))}
        del ws64

    if world == 1 and not args.no_batch:
        line["batched"] = batched_workload(lingam, synth, torch, dev, stream)
        line["batched"]["frac_of_xu_bound"] = {k: v / peak for k, v in line["batched"]["pair_samples_per_s"].items()}

    if world == 1 and args.configs:
        line["configs"] = configs_table(lingam, synth, torch, dev, stream)
    if world == 1 and args.ablation:
        line["ablation"] = ablation(lingam, synth, torch, dev, stream)
    if world == 1 and args.sweep:
        line["scalability_sweep"] = scalability_sweep(lingam, synth, torch, dev, stream)

    if world == 1 and rank == 0 and not args.no_cpu:
        import oracle
        X64 = d.X.astype(np.float32).astype(np.float64)
        rate, dt, m, cores = oracle_rate(X64, args.cpu_seconds)
        # one core: the same FindRoot over a 40-variable subset
        U1 = np.sort(np.random.default_rng(3).choice(p, min(p, 40), replace=False))
        t1 = time.perf_counter()
        oracle.find_root_scores(X64, U1, nthreads=1)
        rate1 = len(U1) * (len(U1) - 1) / 2 * n / (time.perf_counter() - t1)
        line["cpu_baseline"] = {"value": rate, "unit": "pair-samples/s", "cores": cores, "kind": "oracle",
                                "cpu_model": cpu_model(), "single_core_value": rate1,
                                "sample": f"oracle FindRoot (Algorithm 2, every ordered pair) over {m} of the "
                                          f"{p} variables of the same dataset, {dt:.1f} s; single core: 40 "
                                          f"variables"}
    if dist is not None:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--p", type=int, default=P_DEFAULT)
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--fp64-iters", type=int, default=5)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-workload leg")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffer) leg")
    ap.add_argument("--max-iters", type=int, default=0, help="order only the first k iterations (profiling)")
    ap.add_argument("--ablation", action="store_true",
                    help="also time the threshold and the pair reuse switched off (the paper's schedule claims)")
    ap.add_argument("--sweep", action="store_true",
                    help="also run the paper's scalability grid (sparse/dense graphs, p x n)")
    ap.add_argument("--configs", action="store_true",
                    help="also time the five benchmark configurations over dataset seeds 1-5")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()

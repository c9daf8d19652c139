#!/usr/bin/env python
"""Benchmark: Parallel-l0 decodes per second on one GB300 (or N, as replicas).

One step = one complete Parallel-l0 decode (Alg. 2: score all columns, apply,
recompute r and ||r||_0, until the stop rule) of an instance of the workload,
inputs resident in HBM.  Default workload: extreme undersampling (Sec. 5.5
shape, n/m ~ 10^3): n=2^24, m=16777, k=round(0.05 m)=839, d=9, N(0,1)
nonzeros on the 2^-32 grid, uniform support and expander, one instance per
call.  Its CSC alone (604 MB) is far larger than L2, so every iteration
streams it from HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...   # the CPU oracle on the host cores

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank decodes its
own instances (no data exchange) and the value is all ranks' decodes over the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Parallel-l0 decodes/s + HBM GB/s vs peak, batched vs plain; p99 latency"
FALLBACK_HBM_GBS = 6800.0
TABLE3_SECONDS = {22: 0.0167, 24: 0.0557, 26: 0.2319}  # Table 3, K40, rho=0.05, d=7


def workload(name: str, seed: int):
    from paper_1508_01256_gb300 import inputs
    if name == "at-scale":
        return inputs.plain_at_scale(seed=seed)
    if name == "small":
        return inputs.plain_small(seed=seed)
    if name == "extreme":
        return inputs.extreme_undersampling(0.05, d=9, seed=seed)
    if name == "table3":
        return inputs.extreme_undersampling(0.05, d=7, seed=seed)
    raise SystemExit(f"unknown workload {name}")


def workload_config(name: str, p) -> dict:
    """The workload, identical on the GPU arm and the reference arm."""
    return {"workload": {"at-scale": "plain Parallel-l0 at scale",
                         "small": "plain Parallel-l0, single small instance",
                         "extreme": "extreme undersampling n/m ~ 10^3 (rho=0.05, d=9)",
                         "table3": "Table 3 shape (delta=1e-3, rho=0.05, d=7)"}[name],
            "n": p.n, "m": p.m, "k": p.k, "d": p.d, "alpha": 2, "values": p.model,
            "l2": "inputs larger than L2 (CSC alone 4dn bytes); L2 also flushed between "
                  "steps (512 MB write)" if 4 * p.d * p.n > 2 ** 27 else
                  "flushed between steps (512 MB write)"}


def decode_bytes(p, iterations, row_driven=0, row_entries=0) -> float:
    """Algorithmic bytes of one decode.  A column-stream iteration moves 4dn
    (every column's d row indices) + 8m (one read of r by the score) + 16m
    (y and r by the residual); a row-driven iteration moves 4 bytes per CSR
    entry of the nonzero rows (row_entries over all of them) + 24m.  Once:
    8n (writing x_hat) and 16k (the updates of the k support columns, a
    lower bound of the accepted pairs)."""
    return ((iterations - row_driven) * (4 * p.d * p.n + 24 * p.m) + row_driven * 24 * p.m +
            4 * row_entries + 8 * p.n + 16 * p.k)


def vs_baseline(name: str, p, value: float):
    if name == "table3" and p.n in (2 ** 22, 2 ** 24, 2 ** 26):
        return value / (1.0 / TABLE3_SECONDS[p.n.bit_length() - 1])
    return None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        for key in ("hbm_gbs", "hbm_GBps", "hbm"):
            if key in d:
                return float(d[key]), "measured"
    except (OSError, ValueError):
        pass
    return FALLBACK_HBM_GBS, "fallback"


KERNEL_SOURCES = ("ccs_engine_kernel.cuh", "ccs_engine.cu", "ccs_device.cuh", "ccs_internal.cuh")


def kernel_source_sha() -> str:
    """Hash of the sources the persistent engine is compiled from."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1508_01256_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_record(kernel: str, workload_name: str):
    """Per-launch DRAM bytes from a committed ncu summary, if it was taken on
    the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    entry = rec.get(kernel, {}).get(workload_name)
    if not entry:
        return None
    try:
        sha = kernel_source_sha()
    except OSError:
        return None
    return entry["bytes_per_launch"] if sha == entry.get("source_sha") else None


def slowest_over_ranks(times, dist=None, device=None):
    """Each timing's maximum over the ranks of the job (the slowest rank
    defines the job's time); the local values when there is no process group."""
    if dist is None:
        return [float(t) for t in times]
    import torch
    t = torch.tensor([float(x) for x in times], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu().tolist()]


def job_rate(units_per_rank: float, world: int, slowest_s: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (every rank does the same amount of work)."""
    return world * units_per_rank / slowest_s


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples (every 200 ms) from before
    the warm-up to the end of the end-to-end loop, which brackets the timed
    region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.tmp = None

    def __enter__(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.tmp is None:
            return None
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle timing (baseline / reference arm)
# ---------------------------------------------------------------------------

def oracle_instances(name: str, count: int, base_seed: int):
    """`count` instances of the workload for the oracle, generated in
    parallel host threads (the oracle's C routines release the GIL)."""
    import oracle
    insts = [None] * count

    def gen(i):
        p = workload(name, base_seed + i)
        A = oracle.make_expander(p.n, p.m, p.d, p.a_seed)
        y = oracle.measure(A, p.m, p.x)
        insts[i] = (p, A, y)

    threads = [threading.Thread(target=gen, args=(i,)) for i in range(count)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    return insts


def oracle_round(insts):
    """Decode every instance concurrently, one host thread each (the oracle
    itself is single-threaded); returns (wall seconds, all exact)."""
    import numpy as np

    import oracle
    ok = [False] * len(insts)

    def run(i):
        p, A, y = insts[i]
        res = oracle.parallel_l0(A, p.m, y)
        ok[i] = res["status"] == oracle.CONVERGED and np.array_equal(res["x_hat"], p.x)

    threads = [threading.Thread(target=run, args=(i,)) for i in range(len(insts))]
    t0 = time.perf_counter()
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    return time.perf_counter() - t0, all(ok)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(name: str, budget_s: float = 12.0):
    """The oracle as it stands on the host cores: rounds of `cores` concurrent
    single-threaded decodes of distinct instances of the workload, until
    about `budget_s` of wall time (at least one round)."""
    cores = host_cores()
    insts = oracle_instances(name, cores, 777000)
    decodes, elapsed, rounds, exact = 0, 0.0, 0, True
    while rounds == 0 or (elapsed < budget_s and rounds < 8):
        dt, ok = oracle_round(insts)
        elapsed += dt
        decodes += len(insts)
        rounds += 1
        exact &= ok
    return {"value": decodes / elapsed, "unit": "decodes/s", "cores": cores, "kind": "oracle",
            "sample": f"{rounds} round(s) x {cores} concurrent single-threaded oracle decodes "
                      f"of the same workload ({decodes} decodes, {elapsed:.1f} s)",
            "exact_recovery": exact}


def undersampling_sweep(ccs, dev, reps: int, peak: float, seed: int):
    """n/m ~ 10^3 (Sec. 5.5 shape): n=2^24, m=16777, d=9, rho = 0.05..0.30 in
    six steps on gauss-grid values, the +/-1 (non-dissociated) variant at
    rho=0.05 with and without column scaling (Sec. 4.3.3), and d=7,
    rho=0.05 beside the paper's Table 3 time.  Each point:
    one untimed decode, then `reps` decodes with an L2 flush before each,
    timed with CUDA events on the launching stream.  The CSC alone (604 MB at
    d=9) is far larger than L2, so every iteration streams it from HBM."""
    import numpy as np
    import torch

    from paper_1508_01256_gb300 import inputs
    points = [(9, rho, "gauss-grid") for rho in (0.05, 0.10, 0.15, 0.20, 0.25, 0.30)]
    points += [(9, 0.05, "pm1"), (9, 0.05, "pm1-scaled"), (7, 0.05, "gauss-grid")]
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    names = {ccs.CONVERGED: "converged", ccs.STALLED: "stalled", ccs.MAX_ITER: "max_iter"}
    out = []
    for i, (d, rho, model) in enumerate(points):
        scaled = model.endswith("-scaled")
        p = inputs.extreme_undersampling(rho, d=d, seed=seed + i,
                                         model=model.replace("-scaled", ""))
        csc, ptr, cols = ccs.make_expander(p.n, p.m, p.d, p.a_seed, device=dev)
        x_dev = p.x_device(dev)
        if scaled:
            # Sec. 4.3.3: A's columns scaled by i.i.d. numbers; the decode
            # recovers z = s . x and x = z / s
            sc = ccs.column_scales(p.n, seed + 1000 + i, dev)
            y = ccs.measure_scaled(ptr, cols, sc, x_dev, p.m, p.d)
        else:
            y = ccs.measure(ptr, cols, x_dev, p.m, p.d)
        ws = ccs.workspace(ccs.ccs_workspace_size(ccs.OP_DECODE, p.n, p.m, p.d), dev)
        x_hat = torch.empty(p.n, dtype=torch.float64, device=dev)
        r = torch.empty(p.m, dtype=torch.float64, device=dev)
        prm = ccs.params()
        res_dev = ccs.result_buffer(reps + 1, dev)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(reps)]
        for t in range(reps + 1):
            flush.zero_()
            if t > 0:
                evs[t - 1][0].record(stream)
            ccs.ccs_decode_parallel_l0_async(p.n, p.m, p.d, csc, ptr, cols, y, x_hat, r, None,
                                             prm, res_dev[t * ccs.RESULT_BYTES:], ws, stream)
            if t > 0:
                evs[t - 1][1].record(stream)
        torch.cuda.synchronize()
        res = ccs.results_from_device(res_dev, reps + 1)
        ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
        last = res[-1]
        it = last.iterations
        alg = decode_bytes(p, it, last.row_driven, last.row_entries)
        gbs = alg / (ms * 1e-3) / 1e9
        x_out = ccs.unscale(sc, x_hat) if scaled else x_hat
        entry = {"n": p.n, "m": p.m, "d": p.d, "k": p.k, "rho": rho, "values": model,
                 "ms_per_decode": ms, "decodes_per_s": 1000.0 / ms, "iterations": it,
                 "row_driven_iterations": last.row_driven, "row_entries": last.row_entries,
                 "status": names.get(last.status, last.status),
                 "exact_recovery": bool(last.status == ccs.CONVERGED and
                                        torch.equal(x_out, x_dev)),
                 "same_every_rep": all((q.status, q.iterations, q.r0_final) ==
                                       (res[0].status, res[0].iterations, res[0].r0_final)
                                       for q in res),
                 "algorithmic_bytes": alg, "achieved_gbs": gbs, "frac": gbs / peak,
                 "column_updates_per_s": p.n * it / (ms * 1e-3)}
        out.append(entry)
        del csc, ptr, cols, y, ws, x_hat, r, x_dev, x_out
        torch.cuda.empty_cache()
    return {"reps": reps, "l2": "flushed before every decode (512 MB write)",
            "bytes": "per decode: iterations x (4 d n + 24 m) + 8 n + 16 k", "points": out}


def table3_rows(ccs, dev, problems: int, peak: float, seed: int):
    """Table 3's workload at its three sizes: n = 2^22, 2^24, 2^26, delta =
    10^-3, rho = 0.05, d = 7, alpha = 2, `problems` distinct problems per
    size, each decoded alone (CUDA events on the launching stream, L2
    flushed before each).  Mean time of the converged decodes, as the
    paper's table, beside its K40 times (context, not a target)."""
    import torch

    from paper_1508_01256_gb300 import inputs
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rows = []
    for log2n in (22, 24, 26):
        n = 2 ** log2n
        m = inputs.round_half_up(n * 1e-3)
        k = inputs.round_half_up(0.05 * m)
        x_hat = torch.empty(n, dtype=torch.float64, device=dev)
        r = torch.empty(m, dtype=torch.float64, device=dev)
        ws = ccs.workspace(ccs.ccs_workspace_size(ccs.OP_DECODE, n, m, 7), dev)
        prm = ccs.params()
        ms_ok, iters, conv, exact, alg = [], [], 0, 0, []
        for t in range(problems):
            p = inputs.make_problem(n, m, 7, k, seed + 100 * log2n + t)
            csc, ptr, cols = ccs.make_expander(n, m, 7, p.a_seed, device=dev)
            xd = p.x_device(dev)
            y = ccs.measure(ptr, cols, xd, m, 7)
            flush.zero_()
            e0.record(stream)
            res = ccs.ccs_decode_parallel_l0(n, m, 7, csc, ptr, cols, y, x_hat, r, None, prm,
                                             ws, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            iters.append(res.iterations)
            if res.status == ccs.CONVERGED:
                conv += 1
                ms = e0.elapsed_time(e1)
                ms_ok.append(ms)
                alg.append(decode_bytes(p, res.iterations, res.row_driven, res.row_entries) /
                           (ms * 1e-3) / 1e9)
                exact += bool(torch.equal(x_hat, xd))
            del csc, ptr, cols, y, xd
        del x_hat, r, ws
        torch.cuda.empty_cache()
        mean_ms = statistics.mean(ms_ok) if ms_ok else None
        rows.append({"n": n, "m": m, "k": k, "d": 7, "problems": problems, "converged": conv,
                     "exact_recovery": exact, "mean_ms_converged": mean_ms,
                     "mean_iterations": statistics.mean(iters),
                     "mean_achieved_gbs": statistics.mean(alg) if alg else None,
                     "frac": statistics.mean(alg) / peak if alg else None,
                     "paper_k40_s": TABLE3_SECONDS[log2n],
                     "paper_over_this": (TABLE3_SECONDS[log2n] / (mean_ms * 1e-3))
                     if mean_ms else None})
    return {"workload": "Table 3: delta=1e-3, rho=0.05, d=7, alpha=2, gauss-grid",
            "rows": rows}


def alpha_sweep(ccs, dev, seed: int, reps: int = 3):
    """The same n = 2^20 problem decoded with every alpha in [2, d] under both
    scores: the l0 decrease of Eq. (15) and the match count of Alg. 8 (whose
    alpha = floor(d/2) + 1 is Parallel-LDDSR, Sec. 4.3.2), then the shifted
    variant (Sec. 4.3.1) beside Alg. 2 at alpha = 2.  Per setting:
    decodes/s (CUDA events, L2 flushed before each), iterations, outcome."""
    import numpy as np
    import torch

    from paper_1508_01256_gb300 import inputs
    p = inputs.plain_at_scale(seed=seed)
    csc, ptr, cols = ccs.make_expander(p.n, p.m, p.d, p.a_seed, device=dev)
    y = ccs.measure(ptr, cols, p.x_device(dev), p.m, p.d)
    ws = ccs.workspace(ccs.ccs_workspace_size(ccs.OP_DECODE, p.n, p.m, p.d), dev)
    x_hat = torch.empty(p.n, dtype=torch.float64, device=dev)
    r = torch.empty(p.m, dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    names = {ccs.CONVERGED: "converged", ccs.STALLED: "stalled", ccs.MAX_ITER: "max_iter"}
    out = []
    for mode, mode_name in ((ccs.SCORE_L0_DECREASE, "l0_decrease"), (ccs.SCORE_COUNT, "count")):
        for alpha in range(2, p.d + 1):
            prm = ccs.params(alpha=alpha, score_mode=mode)
            res_dev = ccs.result_buffer(reps + 1, dev)
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(reps)]
            for t in range(reps + 1):
                flush.zero_()
                if t > 0:
                    evs[t - 1][0].record(stream)
                ccs.ccs_decode_parallel_l0_async(p.n, p.m, p.d, csc, ptr, cols, y, x_hat, r,
                                                 None, prm, res_dev[t * ccs.RESULT_BYTES:], ws,
                                                 stream)
                if t > 0:
                    evs[t - 1][1].record(stream)
            torch.cuda.synchronize()
            last = ccs.results_from_device(res_dev, reps + 1)[-1]
            ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
            out.append({"score": mode_name, "alpha": alpha,
                        "parallel_lddsr": mode == ccs.SCORE_COUNT and alpha == p.d // 2 + 1,
                        "decodes_per_s": 1000.0 / ms, "iterations": last.iterations,
                        "status": names.get(last.status, last.status),
                        "exact_recovery": bool(last.status == ccs.CONVERGED and
                                               np.array_equal(x_hat.cpu().numpy(), p.x))})
    # the shifted variant (Sec. 4.3.1) at alpha = 2 beside Alg. 2
    for shifted in (False, True):
        prm = ccs.params(shifted=shifted)
        res_dev = ccs.result_buffer(reps + 1, dev)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(reps)]
        for t in range(reps + 1):
            flush.zero_()
            if t > 0:
                evs[t - 1][0].record(stream)
            ccs.ccs_decode_parallel_l0_async(p.n, p.m, p.d, csc, ptr, cols, y, x_hat, r, None,
                                             prm, res_dev[t * ccs.RESULT_BYTES:], ws, stream)
            if t > 0:
                evs[t - 1][1].record(stream)
        torch.cuda.synchronize()
        last = ccs.results_from_device(res_dev, reps + 1)[-1]
        ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
        out.append({"score": "l0_decrease", "alpha": 2, "shifted": shifted,
                    "decodes_per_s": 1000.0 / ms, "iterations": last.iterations,
                    "status": names.get(last.status, last.status),
                    "exact_recovery": bool(last.status == ccs.CONVERGED and
                                           np.array_equal(x_hat.cpu().numpy(), p.x))})
    return {"workload": f"n={p.n}, m={p.m}, d={p.d}, k={p.k}, gauss-grid", "points": out}


def phase_sweep(ccs, dev, seed: int):
    """Sec. 5.1's phase-transition protocol, reduced to run in seconds:
    n = 2^16, d = 7, four deltas, 5 problems per point; then banded signals
    (Sec. 5.6) at delta = 0.1.  rho* is the 50 % point of the logistic fit."""
    from paper_1508_01256_gb300 import phase
    t0 = time.perf_counter()
    res = phase.phase_transition(ccs, n=2 ** 16, d=7, deltas=[0.02, 0.1, 0.3, 0.5],
                                 per_point=5, seed=seed, device=dev)
    bands = [dict(phase.sweep_delta(ccs, 2 ** 16, 7, 0.1, per_point=5, seed=seed + 7,
                                    model="banded", band=b, device=dev), band=b)
             for b in (0.5, 0.9)]
    return {"protocol": "Sec. 5.1: rho from 0.01 in steps of 0.01 while a point recovers; "
                        "logistic 50 % point; n=2^16, d=7, 5 problems per point",
            "deltas": res, "banded_delta_0.1": bands,
            "wall_s": time.perf_counter() - t0}


def batched_vs_plain(ccs, dev, count: int, seed: int, reps: int = 3):
    """Decodes/s of `count` mixed problems (n log-uniform in [2^12, 2^20],
    delta, rho, d drawn from the batched workload's sets) in ONE persistent
    launch, against the same problems as `count` back-to-back plain
    single-problem launches on the same stream.  L2 flushed before each."""
    import torch

    from paper_1508_01256_gb300 import inputs
    probs = inputs.batch_problems(count, seed=seed)
    items, pbs, outs = [], [], []
    for p in probs:
        csc, ptr, cols = ccs.make_expander(p.n, p.m, p.d, p.a_seed, device=dev)
        y = ccs.measure(ptr, cols, torch.from_numpy(p.x).to(dev), p.m, p.d)
        x_hat = torch.empty(p.n, dtype=torch.float64, device=dev)
        r = torch.empty(p.m, dtype=torch.float64, device=dev)
        items.append((p, csc, ptr, cols, y))
        outs.append((x_hat, r))
        pbs.append(ccs.problem(csc, ptr, cols, y, x_hat, r))
    ws_b = ccs.workspace(ccs.ccs_batch_workspace_size(pbs), dev)
    ws_p = ccs.workspace(max(ccs.ccs_workspace_size(ccs.OP_DECODE, p.n, p.m, p.d) for p in probs), dev)
    res_b = ccs.result_buffer(count, dev)
    res_p = ccs.result_buffer(count, dev)
    prm = ccs.params()
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    # launch shapes of the batched launches picked by the library's
    # autotuner (untimed); the plain single-problem launches keep the rule
    tuned = ccs.ccs_autotune(pbs, prm, ws_b, stream)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    tb, tp = [], []
    for rep in range(reps + 1):
        flush.zero_()
        ev[0].record(stream)
        ccs.ccs_decode_batch_async(pbs, prm, res_b, ws_b, stream)
        ev[1].record(stream)
        torch.cuda.synchronize()
        if rep:
            tb.append(ev[0].elapsed_time(ev[1]))
        flush.zero_()
        ev[0].record(stream)
        for i, (p, csc, ptr, cols, y) in enumerate(items):
            x_hat, r = outs[i]
            ccs.ccs_decode_parallel_l0_async(p.n, p.m, p.d, csc, ptr, cols, y, x_hat, r, None,
                                             prm, res_p[i * ccs.RESULT_BYTES:], ws_p, stream)
        ev[1].record(stream)
        torch.cuda.synchronize()
        if rep:
            tp.append(ev[0].elapsed_time(ev[1]))
    # the same batch captured once in a CUDA graph and replayed
    graph = ccs.BatchGraph(pbs, prm, dev)
    tg = []
    for rep in range(reps + 1):
        flush.zero_()
        ev[0].record(stream)
        graph.launch(stream)
        ev[1].record(stream)
        torch.cuda.synchronize()
        if rep:
            tg.append(ev[0].elapsed_time(ev[1]))
    rg = graph.read_results()
    graph.close()
    # the converging problems alone (the max_iter tail excluded), as one batch
    rb0 = ccs.results_from_device(res_b, count)
    conv_idx = [i for i, a in enumerate(rb0) if a.status == ccs.CONVERGED]
    conv_pbs = [pbs[i] for i in conv_idx]
    ws_c = ccs.workspace(ccs.ccs_batch_workspace_size(conv_pbs), dev)
    res_c = ccs.result_buffer(len(conv_pbs), dev)
    tc = []
    for rep in range(reps + 1):
        flush.zero_()
        ev[0].record(stream)
        ccs.ccs_decode_batch_async(conv_pbs, prm, res_c, ws_c, stream)
        ev[1].record(stream)
        torch.cuda.synchronize()
        if rep:
            tc.append(ev[0].elapsed_time(ev[1]))
    rc_ = ccs.results_from_device(res_c, len(conv_pbs))
    mc = statistics.median(tc)
    alg_c = sum(a.iterations * (4 * probs[i].d * probs[i].n + 8 * probs[i].m)
                for i, a in zip(conv_idx, rc_))
    del ws_c
    ccs.ccs_autotune_reset()
    rb = ccs.results_from_device(res_b, count)
    rp = ccs.results_from_device(res_p, count)
    same = all(a.status == b.status == c.status and a.iterations == b.iterations == c.iterations
               and a.r0_final == b.r0_final == c.r0_final for a, b, c in zip(rb, rp, rg))
    conv = sum(a.status == ccs.CONVERGED for a in rb)
    exact = sum(a.status == ccs.CONVERGED and bool((outs[i][0].cpu().numpy() == items[i][0].x).all())
                for i, a in enumerate(rb))
    mb, mp, mg = statistics.median(tb), statistics.median(tp), statistics.median(tg)
    cols_total = sum(p.n * a.iterations for p, a in zip(probs, rb))
    # aggregate roofline of the batched launch: every problem's algorithmic
    # bytes, iterations x (4 d n + 8 m), over the batched time
    alg = sum(a.iterations * (4 * p.d * p.n + 8 * p.m) for p, a in zip(probs, rb))
    peak = measured_peaks()[0]
    return {"problems": count, "batched_decodes_per_s": count / (mb / 1000.0),
            "algorithmic_bytes": alg, "achieved_gbs": alg / (mb * 1e-3) / 1e9,
            "frac": alg / (mb * 1e-3) / 1e9 / peak,
            "plain_decodes_per_s": count / (mp / 1000.0), "batched_ms": mb, "plain_ms": mp,
            "graph_batched_decodes_per_s": count / (mg / 1000.0), "graph_ms": mg,
            "speedup": mp / mb, "batched_column_updates_per_s": cols_total / (mb / 1000.0),
            "autotuned_shapes": [t for t in tuned if t],
            "converging_only": {"problems": len(conv_pbs),
                                "decodes_per_s": len(conv_pbs) / (mc / 1000.0), "ms": mc,
                                "achieved_gbs": alg_c / (mc * 1e-3) / 1e9,
                                "frac": alg_c / (mc * 1e-3) / 1e9 / measured_peaks()[0]},
            "same_results": same, "converged": conv, "exact_recovery": exact,
            "max_iterations": max(a.iterations for a in rb),
            "workload": "n log-uniform 2^12..2^20, m/n in {0.01,0.05,0.1,0.3}, "
                        "k/m in {0.05,0.1,0.2}, d in {5,7,9,11}, gauss-grid; launch shapes "
                        "autotuned (1: 1024 threads, 2: 512, 3: 768 a CTA)"}


SERVE_LOADS = (0.5, 0.6, 0.7, 0.8, 0.9, 1.0)


def serving_run(ccs, dev, count: int, seed: int, pool_bytes: int = 16 << 30,
                max_batch: int = 512, iters_per_round: int = 2, oracle_checks: int = 6):
    """Serving workload (config 5) with seeded requests: `count` distinct
    requests, n log-uniform 2^12..2^22, delta and rho as in the batched
    workload, d in {7, 9}.  Each request hands the server its expander seed
    and host y; the server draws A into its pool at admission, decodes, and
    copies x_hat back to a host buffer, so the pool (`pool_bytes`) bounds
    every byte a request holds on the device.  First a closed-loop burst of
    a sixth of the requests gives the peak decodes/s; then the rest arrive
    as open-loop Poisson streams at each load in SERVE_LOADS x that peak,
    an equal share per load, each on a fresh server.  Latency = host buffer
    filled - submission, from the library's clock.  Every result is checked
    for exact recovery against x; a sample is decoded alone on the GPU and
    the smallest ones by the oracle, bit for bit."""
    import random

    import numpy as np
    import torch

    from paper_1508_01256_gb300 import inputs
    t_setup = time.perf_counter()
    shapes = inputs.batch_shapes(count, seed=seed, log2n_hi=22.0, ds=(7, 9))
    probs, reqs = [], []
    for q, (n, m, d, k) in enumerate(shapes):
        p = inputs.make_problem(n, m, d, k, seed * 7919 + q)
        csc, ptr, cols = ccs.make_expander(p.n, p.m, p.d, p.a_seed, device=dev)
        y = ccs.measure(ptr, cols, p.x_device(dev), p.m, p.d).cpu().numpy()
        probs.append(p)
        reqs.append((p.n, p.m, p.d, p.a_seed, y))
        del csc, ptr, cols
    torch.cuda.empty_cache()
    setup_s = time.perf_counter() - t_setup
    rng = random.Random(seed)
    keep = set(rng.sample(range(count), min(12, count)))
    small = [q for q in range(count) if probs[q].n <= 2 ** 15]
    oracle_q = set(rng.sample(small, min(oracle_checks, len(small))))
    kept = {}
    tally = {"converged": 0, "exact": 0}

    def on_done(q, info, out):
        # out: x_hat's nonzeros (indices ascending, values, count)
        p = probs[q]
        idx, val, nnz = out
        ok = info.result.status == ccs.CONVERGED and info.result.error == 0
        tally["converged"] += ok
        tally["exact"] += bool(ok and nnz[0] == p.k and np.array_equal(idx[:p.k], p.idx) and
                               np.array_equal(val[:p.k], p.val))
        if q in keep or q in oracle_q:
            x_hat = np.zeros(p.n)
            take = min(int(nnz[0]), idx.size)
            x_hat[idx[:take]] = val[:take]
            kept[q] = (info.result, x_hat, int(nnz[0]))

    def run(qs, arrivals):
        timeline = []
        with ccs.Server(pool_bytes, max_batch=max_batch, iters_per_round=iters_per_round) as srv:
            infos = ccs.serve_seeded(srv, [reqs[q] for q in qs], arrivals,
                                     lambda i, info, x: on_done(qs[i], info, x),
                                     sampler=timeline,
                                     nonzeros_cap=lambda i: 2 * probs[qs[i]].k + 64)
            st = srv.stats()
        lat = sorted(1000.0 * (i.done_s - i.submit_s) for i in infos)
        conv = sorted(1000.0 * (i.done_s - i.submit_s) for i in infos
                      if i.result.status == ccs.CONVERGED)

        def pct(v, f):
            return v[min(len(v) - 1, int(f * len(v)))] if v else None
        span = max(i.done_s for i in infos) - min(i.submit_s for i in infos)
        infl = [t[1] for t in timeline]
        step = max(1, len(timeline) // 16)
        return {"requests": len(qs), "decodes_per_s": len(qs) / span,
                "p50_ms": pct(lat, 0.5), "p99_ms": pct(lat, 0.99), "max_ms": lat[-1],
                "converged_requests": len(conv), "p50_ms_converged": pct(conv, 0.5),
                "p99_ms_converged": pct(conv, 0.99), "rounds": st["rounds"],
                "peak_inflight": st["peak_inflight"], "peak_pool_bytes": st["peak_bytes"],
                "mean_inflight": statistics.mean(infl) if infl else None,
                "inflight_over_time": [(round(t[0], 4), t[1], t[2]) for t in timeline[::step]],
                "errors": sum(i.result.error != 0 for i in infos)}

    n_closed = max(1, count // 6)
    closed_q = list(range(n_closed))
    closed = run(closed_q, [0.0] * n_closed)
    peak = closed["decodes_per_s"]
    rest = list(range(n_closed, count))
    per = max(1, len(rest) // len(SERVE_LOADS))
    points = []
    arr_rng = np.random.default_rng(seed + 1)
    for li, load in enumerate(SERVE_LOADS):
        qs = rest[li * per:(li + 1) * per] if li < len(SERVE_LOADS) - 1 else rest[li * per:]
        if not qs:
            break
        arrivals = np.cumsum(arr_rng.exponential(1.0 / (load * peak), size=len(qs)))
        pt = run(qs, arrivals)
        pt.update(load=load, offered_rate_per_s=load * peak)
        points.append(pt)
    # each sampled result equals the same decode alone on the GPU, and the
    # smallest ones the oracle's decode, bit for bit
    same_alone = True
    for q in sorted(keep):
        p = probs[q]
        res, x_hat, nnz = kept[q]
        csc, ptr, cols = ccs.make_expander(p.n, p.m, p.d, p.a_seed, device=dev)
        alone = ccs.decode_parallel_l0(csc, ptr, cols, torch.from_numpy(reqs[q][4]).to(dev),
                                       history=False)
        xa = alone.x_hat.cpu().numpy()
        same_alone &= (res.status, res.iterations, res.r0_final) == \
            (alone.status, alone.iterations, alone.r0_final)
        same_alone &= nnz == int(np.count_nonzero(xa))
        # all nonzeros when the list held them, else the ones returned
        got = np.nonzero(x_hat)[0]
        same_alone &= bool(np.array_equal(x_hat, xa) if nnz <= 2 * p.k + 64
                           else np.array_equal(x_hat[got], xa[got]))
        del csc, ptr, cols, alone
    same_oracle = None
    if oracle_q:
        import oracle
        same_oracle = True
        for q in sorted(oracle_q):
            p = probs[q]
            res, x_hat, nnz = kept[q]
            A = oracle.make_expander(p.n, p.m, p.d, p.a_seed)
            ref = oracle.parallel_l0(A, p.m, reqs[q][4])
            same_oracle &= (res.status, res.iterations, res.r0_final) == \
                (ref["status"], ref["iterations"], ref["r0_final"])
            same_oracle &= nnz == int(np.count_nonzero(ref["x_hat"]))
            got = np.nonzero(x_hat)[0]
            same_oracle &= bool(
                np.array_equal(x_hat.view(np.int64), ref["x_hat"].view(np.int64))
                if nnz <= 2 * p.k + 64 else
                np.array_equal(x_hat[got].view(np.int64), ref["x_hat"][got].view(np.int64)))
    torch.cuda.empty_cache()
    return {"requests": count, "distinct": True, "pool_bytes": pool_bytes,
            "max_batch": max_batch, "iters_per_round": iters_per_round,
            "closed_loop": closed, "peak_decodes_per_s": peak, "load_sweep": points,
            "converged": tally["converged"], "exact_recovery": tally["exact"],
            "same_as_alone_sample": same_alone, "sample_size": len(keep),
            "same_as_oracle_sample": same_oracle, "oracle_sample_size": len(oracle_q),
            "setup_s": setup_s,
            "results": "x_hat as its nonzeros (list of 2k + 64 entries)",
            "workload": "seeded requests (the server draws A from the seed into its pool): "
                        "n log-uniform 2^12..2^22, m/n in {0.01,0.05,0.1,0.3}, k/m in "
                        "{0.05,0.1,0.2}, d in {7,9}, gauss-grid; closed-loop burst of "
                        "count/6, then Poisson arrivals at 0.5-1.0x its rate"}


def run_reference(args):
    from paper_1508_01256_gb300 import inputs  # noqa: F401  (inputs only)
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = host_cores()
    insts = oracle_instances(args.workload, cores, 555000)
    for _ in range(args.warmup):
        oracle_round(insts)
    total, exact = 0.0, True
    for _ in range(args.steps):
        dt, ok = oracle_round(insts)
        total += dt
        exact &= ok
    decodes = args.steps * len(insts)
    value = decodes / total
    p = insts[0][0]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "decodes/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": vs_baseline(args.workload, p, value),
            "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(args.workload, p),
                           parallelism=f"replicas{args.gpus}"),
            "e2e": {"value": value, "unit": "decodes/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "cpu_baseline": {"value": value, "unit": "decodes/s", "cores": cores,
                             "kind": "oracle",
                             "sample": f"each step: {cores} concurrent single-threaded oracle "
                                       f"decodes of distinct instances of the workload, one "
                                       f"per host thread (instance generation untimed)"},
            "decodes_per_step": cores, "exact_recovery": exact, "gpu_launches": 0}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_ccs(args):
    import numpy as np
    import torch

    from paper_1508_01256_gb300 import build as libbuild
    from paper_1508_01256_gb300 import ccs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    libbuild.build()
    ccs.lib()

    # instances resident in HBM
    insts = []
    for i in range(args.instances):
        p = workload(args.workload, 1000 * rank + 17 + i)
        csc, ptr, cols = ccs.make_expander(p.n, p.m, p.d, p.a_seed, device=dev)
        y = ccs.measure(ptr, cols, p.x_device(dev), p.m, p.d)
        insts.append((p, csc, ptr, cols, y))
    p0 = insts[0][0]
    ws = ccs.workspace(ccs.ccs_workspace_size(ccs.OP_DECODE, p0.n, p0.m, p0.d), dev)
    x_hat = torch.empty(p0.n, dtype=torch.float64, device=dev)
    r = torch.empty(p0.m, dtype=torch.float64, device=dev)
    hist = None  # the optional ||r||_0 history is not requested in the timed loop
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)  # > L2 (126 MB)
    stream = torch.cuda.current_stream(dev)

    def decode(i):
        p, csc, ptr, cols, y = insts[i % len(insts)]
        return ccs.decode_parallel_l0(csc, ptr, cols, y, engine=args.engine, ws=ws,
                                      out=(x_hat, r, hist))

    clk = ClockSampler(local).__enter__()
    time.sleep(0.3)  # let nvidia-smi start sampling before the GPU work
    for i in range(args.warmup):
        flush.zero_()
        decode(i)
    torch.cuda.synchronize()

    # timed region: each step enqueues an L2 flush (outside the events) and
    # one asynchronous decode; the host never waits inside the loop
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    res_dev = ccs.result_buffer(args.steps, dev)
    prm = ccs.params(engine=args.engine, schedule=args.schedule)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = ccs.ccs_launch_count()
    ccs.ccs_profile_begin()
    t0 = time.perf_counter()
    for i in range(args.steps):
        p_, csc, ptr, cols, y = insts[i % len(insts)]
        flush.zero_()
        evs[i][0].record(stream)
        ccs.ccs_decode_parallel_l0_async(p_.n, p_.m, p_.d, csc, ptr, cols, y, x_hat, r, None, prm,
                                         res_dev[i * ccs.RESULT_BYTES:], ws, stream)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ktimes = ccs.ccs_profile_end()
    launches = ccs.ccs_launch_count() - launches0
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = [a_.elapsed_time(b_) for a_, b_ in evs]
    total_s = sum(step_ms) / 1000.0
    results = ccs.results_from_device(res_dev, args.steps)
    iters = [rr.iterations for rr in results]
    exact = all(rr.status == ccs.CONVERGED and rr.error == 0 for rr in results)
    # exactness of the last decode of each instance
    for i in range(len(insts)):
        o = decode(args.steps + i)
        exact &= bool(np.array_equal(o.x_hat.cpu().numpy(), insts[(args.steps + i) % len(insts)][0].x))
    # per-phase device times from a few profiled blocking decodes
    ccs.ccs_profile_begin()
    for i in range(min(10, args.steps)):
        flush.zero_()
        decode(i)
    phase_times = ccs.ccs_profile_end()
    for key in ("score", "residual", "score.fingerprints", "score.stream", "score.queue"):
        if key in phase_times:
            ktimes[key] = phase_times[key]

    # end to end through the public API: pinned host inputs -> device, decode,
    # x_hat back to the host, every step
    p, csc, ptr, cols, y = insts[0]
    h_csc, h_ptr, h_cols, h_y = (t.cpu().pin_memory() for t in (csc, ptr, cols, y))
    d_csc, d_ptr, d_cols, d_y = (torch.empty_like(t) for t in (csc, ptr, cols, y))
    h_x = torch.empty(p.n, dtype=torch.float64).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in (h_csc, h_ptr, h_cols, h_y))
    d2h = h_x.numel() * h_x.element_size()
    e2e_steps = max(3, args.steps // 2)
    torch.cuda.synchronize()
    e2e_t = 0.0
    for i in range(e2e_steps + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for dst, src in ((d_csc, h_csc), (d_ptr, h_ptr), (d_cols, h_cols), (d_y, h_y)):
            dst.copy_(src, non_blocking=True)
        o = ccs.decode_parallel_l0(d_csc, d_ptr, d_cols, d_y, engine=args.engine, ws=ws,
                                   out=(x_hat, r, hist))
        h_x.copy_(o.x_hat, non_blocking=True)
        torch.cuda.synchronize()
        if i > 0:  # first pass is a warm-up
            e2e_t += time.perf_counter() - t1
    clk.__exit__(None, None, None)

    # max over ranks
    decodes = args.steps
    total_s, e2e_t = slowest_over_ranks([total_s, e2e_t], dist, dev)
    value = job_rate(decodes, world, total_s)
    e2e_value = job_rate(e2e_steps, world, e2e_t)

    # roofline of the dominant kernel, the persistent launch that runs a
    # whole decode: its algorithmic bytes are decode_bytes() of the mean
    # iteration count.  The score phase alone moves 4 d n + 8 m per iteration.
    per_iter = 4 * p0.d * p0.n + 8 * p0.m
    peak, peak_kind = measured_peaks()
    roof = None
    main = "persistent" if "persistent" in ktimes else "score"
    launches_k, ms_k = ktimes.get(main, (0, 0.0))
    if launches_k:
        avg_s = ms_k / launches_k / 1000.0
        bytes_per_launch = (statistics.mean(decode_bytes(p0, rr.iterations, rr.row_driven,
                                                         rr.row_entries) for rr in results)
                            if main == "persistent" else per_iter)
        achieved = bytes_per_launch / avg_s / 1e9
        roof = {"bound": "hbm", "kernel": main, "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
                "traffic": traffic_record(main, args.workload),
                "algorithmic_bytes_per_launch": bytes_per_launch,
                "avg_launch_us": avg_s * 1e6}
        sc_n, sc_ms = ktimes.get("score", (0, 0.0))
        if sc_n:
            sc_avg = sc_ms / sc_n / 1000.0
            roof["score_phase"] = {"achieved": per_iter / sc_avg / 1e9,
                                   "frac": per_iter / sc_avg / 1e9 / peak,
                                   "avg_us": sc_avg * 1e6, "count": sc_n}
            for sub in ("score.fingerprints", "score.stream", "score.queue"):
                n_, ms_ = ktimes.get(sub, (0, 0.0))
                if n_:
                    roof["score_phase"][sub.split(".")[1] + "_us"] = 1000.0 * ms_ / n_
    kernel_share = {k: {"launches": v[0], "ms": round(v[1], 4)} for k, v in ktimes.items()}

    batched = None
    if args.batch > 0:
        batched = batched_vs_plain(ccs, dev, args.batch, seed=1000 * rank + 4242)
    serving = None
    if args.serve > 0:
        serving = serving_run(ccs, dev, args.serve, seed=1000 * rank + 777)
    alphas = None
    if args.alpha_sweep > 0:
        alphas = alpha_sweep(ccs, dev, seed=1000 * rank + 31)
    phases = None
    if args.phase > 0:
        phases = phase_sweep(ccs, dev, seed=1000 * rank + 51)
    sweep = None
    if args.undersampling > 0:
        sweep = undersampling_sweep(ccs, dev, args.undersampling, measured_peaks()[0],
                                    seed=1000 * rank + 20151508)
    table3 = None
    if args.table3 > 0:
        table3 = table3_rows(ccs, dev, args.table3, measured_peaks()[0],
                             seed=1000 * rank + 3003)

    if rank == 0:
        cb = None
        if world == 1 and not args.no_cpu_baseline:
            cb = cpu_baseline(args.workload)
        line = {"metric": METRIC, "value": value, "unit": "decodes/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1000.0 * total_s / decodes, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": vs_baseline(args.workload, p0, value),
                "dtype": "f64", "data": "synthetic",
                "config": dict(workload_config(args.workload, p0),
                               parallelism=f"replicas{world}"),
                "launch": {"engine": args.engine, "schedule": args.schedule},
                "decodes_per_step": 1,
                "e2e": {"value": e2e_value, "unit": "decodes/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": launches,
                "roofline": roof,
                "cpu_baseline": cb,
                "clocks": clk.summary(),
                "column_updates_per_s": value * p0.n * statistics.mean(iters),
                "iterations_mean": statistics.mean(iters),
                "row_driven_iterations_mean": statistics.mean(rr.row_driven for rr in results),
                "row_entries_mean": statistics.mean(rr.row_entries for rr in results),
                "exact_recovery": exact,
                "kernel_times": kernel_share,
                "batched": batched,
                "serving": serving,
                "undersampling": sweep,
                "table3": table3,
                "alpha_sweep": alphas,
                "phase_transition": phases,
                "wall_s_timed_region": wall}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ccs", choices=["ccs", "reference"])
    ap.add_argument("--workload", default="extreme",
                    choices=["at-scale", "small", "extreme", "table3"])
    ap.add_argument("--engine", type=int, default=0)
    ap.add_argument("--schedule", type=int, default=0,
                    help="persistent-engine launch shape (0: library's choice)")
    ap.add_argument("--instances", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch", type=int, default=512,
                    help="problems in the batched-vs-plain comparison (0: skip)")
    ap.add_argument("--serve", type=int, default=10000,
                    help="distinct seeded requests in the serving run: a closed-loop sixth, "
                         "the rest over the Poisson load sweep (0: skip)")
    ap.add_argument("--alpha-sweep", type=int, default=1,
                    help="alpha in [2, d] under both scores at n = 2^20 (0: skip)")
    ap.add_argument("--phase", type=int, default=1,
                    help="reduced phase-transition sweep (0: skip)")
    ap.add_argument("--undersampling", type=int, default=3,
                    help="timed decodes per point of the n/m ~ 10^3 sweep (0: skip)")
    ap.add_argument("--table3", type=int, default=30,
                    help="problems per size of the Table 3 rows, n = 2^22, 2^24, 2^26 (0: skip)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ccs(args)


if __name__ == "__main__":
    main()

"""Recovery experiments of Parallel-l0 on the GPU (Sec. 5.1, 5.5, 5.6, 5.7).

Sec. 5.1 (phase transitions): for each delta = m/n, start at rho = k/m = 0.01,
decode a few random problems per point and raise rho by 0.01 while at least
one of them is recovered; fit a logistic curve to the recovery data and
report its 50 % point rho*(delta).  Here every point's problems go to the
GPU as one batched decode (the points of a delta are sent in chunks; the
stopping rule is applied to the collected data, so the data equal those of
the sequential protocol).  Recovery is the outcome CONVERGED with x_hat == x
(on the default gauss-grid values every sum is exact, so this is the
paper's 1e-6 tolerance with nothing to round).

When the recovery data are completely separated (every problem recovered up
to some rho, none beyond), the logistic likelihood has no maximum: its slope
grows without bound.  The transition is then reported as that bracket, not
as a fitted number.

Sec. 5.5 (small delta): delta = 10^-3, d = 7, rho from 0.01 in steps of
0.01, 30 problems per rho, each decoded alone and timed; the sweep goes on
while at least half of a point's problems converge.

Banded signals (Sec. 5.6): the Sec. 5.1 sweep with a fraction `band` of the
support sharing one value.  Sec. 5.7: the same sweep for several d.

    python -m paper_1508_01256_gb300.phase low-delta --log2n 22 24 [--d 7]
    python -m paper_1508_01256_gb300.phase phase [--n-log2 18] [--d 7 ...]
"""
from __future__ import annotations

import math
import statistics

import numpy as np

from . import inputs


def paper_deltas() -> list[float]:
    """delta_p of Sec. 5.1: {0.02 p : p in [4]} u {0.1 + 89/1900 (p - 1) : p in [20]}."""
    return [0.02 * p for p in range(1, 5)] + [0.1 + 89.0 / 1900.0 * (p - 1) for p in range(1, 21)]


def logistic_fit(rho: np.ndarray, success: np.ndarray, iters: int = 100):
    """Maximum-likelihood fit of P(success | rho) = 1 / (1 + exp(b (rho - c)))
    by Newton's method on (b0, b1) of the linear predictor b0 + b1 rho.
    Returns (c, b): the 50 % point and the slope; c is nan when the data do
    not bracket a transition (all successes or all failures)."""
    rho = np.asarray(rho, dtype=np.float64)
    yv = np.asarray(success, dtype=np.float64)
    if yv.size == 0 or yv.min() == yv.max():
        return float("nan"), float("nan")
    X = np.stack([np.ones_like(rho), rho], axis=1)
    w = np.zeros(2)
    for _ in range(iters):
        eta = np.clip(X @ w, -40.0, 40.0)
        p = 1.0 / (1.0 + np.exp(-eta))
        g = X.T @ (yv - p)
        H = (X * (p * (1.0 - p))[:, None]).T @ X + 1e-9 * np.eye(2)
        step = np.linalg.solve(H, g)
        w = w + step
        if np.max(np.abs(step)) < 1e-12:
            break
    b0, b1 = w
    if b1 == 0.0:
        return float("nan"), float("nan")
    return float(-b0 / b1), float(-b1)


def transition(rho, success) -> dict:
    """The 50 % point of recovery data.  Completely separated data (the
    largest rho with a success below the smallest rho with a failure), or
    data whose successes and failures meet at a single rho, have no
    logistic maximum-likelihood fit: the transition is then that bracket
    [lo, hi], rho_star its midpoint, method "bracket".  Otherwise the
    logistic fit (method "logistic"); "none" when the data hold only
    successes or only failures."""
    rho = np.asarray(rho, dtype=np.float64)
    yv = np.asarray(success, dtype=bool)
    if yv.size == 0 or yv.all() or not yv.any():
        return {"rho_star": float("nan"), "slope": float("nan"), "bracket": None,
                "method": "none"}
    lo, hi = float(rho[yv].max()), float(rho[~yv].min())
    if lo <= hi:
        # no failure below the last success: (quasi-)complete separation
        return {"rho_star": 0.5 * (lo + hi), "slope": float("inf"), "bracket": [lo, hi],
                "method": "bracket"}
    c, b = logistic_fit(rho, yv.astype(np.float64))
    return {"rho_star": c, "slope": b, "bracket": None, "method": "logistic"}


def sweep_delta(ccs, n: int, d: int, delta: float, per_point: int = 10, rho_step: float = 0.01,
                chunk: int = 8, seed: int = 20151508, model: str = "gauss-grid",
                band: float = 0.0, max_rho: float = 1.0, device="cuda") -> dict:
    """Recovery data of one delta (Sec. 5.1 protocol) and its logistic rho*."""
    import torch

    m = max(d, inputs.round_half_up(delta * n))
    data = []  # (rho, recovered)
    step = 0
    done = False
    while not done:
        rhos = [rho_step * (step + c + 1) for c in range(chunk)]
        rhos = [r for r in rhos if r <= max_rho + 1e-12]
        if not rhos:
            break
        probs, items = [], []
        for ci, rho in enumerate(rhos):
            k = inputs.round_half_up(rho * m)
            for t in range(per_point):
                p = inputs.make_problem(n, m, d, k, seed + 7919 * (step + ci) + t, model, band)
                csc, ptr, cols = ccs.make_expander(n, m, d, p.a_seed, device=device)
                y = ccs.measure(ptr, cols, p.x_device(device), m, d)
                probs.append(p)
                items.append((csc, ptr, cols, y))
        outs = ccs.decode_batch(items)
        for ci, rho in enumerate(rhos):
            ok = 0
            for t in range(per_point):
                q = ci * per_point + t
                rec = outs[q].status == ccs.CONVERGED and bool(
                    torch.equal(outs[q].x_hat, probs[q].x_device(device)))
                data.append((rho, rec))
                ok += rec
            if ok == 0:  # the protocol stops at the first point with no recovery
                done = True
                break
        step += len(rhos)
        del items, outs
    rho_arr = np.array([r for r, _ in data])
    suc = np.array([s for _, s in data], dtype=np.float64)
    tr = transition(rho_arr, suc)
    return {"delta": delta, "m": m, "n": n, "d": d, "rho_star": tr["rho_star"],
            "slope": tr["slope"], "bracket": tr["bracket"], "method": tr["method"],
            "points": len(data) // per_point, "recovered": int(suc.sum()),
            "decodes": int(suc.size)}


def phase_transition(ccs, n: int = 2 ** 18, d: int = 7, deltas=None, per_point: int = 10,
                     seed: int = 20151508, model: str = "gauss-grid", band: float = 0.0,
                     device="cuda") -> list[dict]:
    """rho*(delta) for each delta (default: the paper's 24 values)."""
    deltas = paper_deltas() if deltas is None else list(deltas)
    return [sweep_delta(ccs, n, d, dl, per_point=per_point, seed=seed + 101 * i, model=model,
                        band=band, device=device) for i, dl in enumerate(deltas)]


def low_delta_protocol(ccs, log2n: int, d: int = 7, delta: float = 1e-3, per_point: int = 30,
                       rho_step: float = 0.01, seed: int = 20151508, max_rho: float = 1.0,
                       score_mode: int = 0, alpha: int = 2, device="cuda") -> dict:
    """Sec. 5.5 at one n: rho = 0.01, 0.02, ... with `per_point` problems
    each, every problem decoded alone and timed (CUDA events on the launching
    stream, L2 flushed before each decode); the sweep goes on while at least
    half of a point's problems converge.  Per point: converged and exactly
    recovered counts, iterations, and the mean time of the converged decodes
    (the quantity of the paper's figure on delta = 0.001).  rho_50 is the
    last rho at which at least half converged."""
    import torch

    n = 2 ** log2n
    m = max(d, inputs.round_half_up(delta * n))
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=device)
    stream = torch.cuda.current_stream(device)
    x_hat = torch.empty(n, dtype=torch.float64, device=device)
    r = torch.empty(m, dtype=torch.float64, device=device)
    ws = ccs.workspace(ccs.ccs_workspace_size(ccs.OP_DECODE, n, m, d), device)
    prm = ccs.params(alpha=alpha, score_mode=score_mode)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    points, data = [], []
    step = 1
    while rho_step * step <= max_rho + 1e-12:
        rho = round(rho_step * step, 10)
        k = inputs.round_half_up(rho * m)
        conv, exact, ms_ok, iters = 0, 0, [], []
        statuses = {}
        for t in range(per_point):
            p = inputs.make_problem(n, m, d, k, seed + 1000003 * step + t)
            csc, ptr, cols = ccs.make_expander(n, m, d, p.a_seed, device=device)
            xd = p.x_device(device)
            y = ccs.measure(ptr, cols, xd, m, d)
            flush.zero_()
            e0.record(stream)
            res = ccs.ccs_decode_parallel_l0(n, m, d, csc, ptr, cols, y, x_hat, r, None, prm,
                                             ws, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            ok = res.status == ccs.CONVERGED
            rec = ok and bool(torch.equal(x_hat, xd))
            conv += ok
            exact += rec
            iters.append(res.iterations)
            statuses[ccs.STATUS_NAMES[res.status]] = statuses.get(
                ccs.STATUS_NAMES[res.status], 0) + 1
            if ok:
                ms_ok.append(ms)
            data.append((rho, rec))
            del csc, ptr, cols, y, xd
        points.append({"rho": rho, "k": k, "converged": conv, "exact": exact,
                       "problems": per_point, "outcomes": statuses,
                       "mean_ms_converged": statistics.mean(ms_ok) if ms_ok else None,
                       "mean_iterations": statistics.mean(iters)})
        if 2 * conv < per_point:
            break
        step += 1
    tr = transition([a for a, _ in data], [b for _, b in data])
    last_ok = [q["rho"] for q in points if 2 * q["converged"] >= per_point]
    return {"n": n, "m": m, "d": d, "delta": delta, "alpha": alpha,
            "score": "count" if score_mode else "l0_decrease", "per_point": per_point,
            "rho_50": last_ok[-1] if last_ok else None, "fit": tr, "points": points}


def _main(argv=None):
    import argparse
    import json

    import torch

    from . import build, ccs
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    lo = sub.add_parser("low-delta", help="Sec. 5.5: delta = 1e-3 sweep per n")
    lo.add_argument("--log2n", type=int, nargs="+", default=[22, 24])
    lo.add_argument("--d", type=int, default=7)
    lo.add_argument("--per-point", type=int, default=30)
    lo.add_argument("--alpha", type=int, default=2)
    lo.add_argument("--score", choices=["l0_decrease", "count"], default="l0_decrease")
    ph = sub.add_parser("phase", help="Sec. 5.1 / 5.7: rho*(delta) at each d")
    ph.add_argument("--n-log2", type=int, default=18)
    ph.add_argument("--d", type=int, nargs="+", default=[7])
    ph.add_argument("--per-point", type=int, default=10)
    ph.add_argument("--deltas", type=float, nargs="*", default=None)
    ph.add_argument("--band", type=float, nargs="*", default=None,
                    help="Sec. 5.6: banded signals with these fractions of equal values")
    ap.add_argument("--seed", type=int, default=20151508)
    args = ap.parse_args(argv)
    build.build()
    dev = torch.device("cuda", 0)
    if args.cmd == "low-delta":
        for lg in args.log2n:
            out = low_delta_protocol(ccs, lg, d=args.d, per_point=args.per_point,
                                     alpha=args.alpha, seed=args.seed,
                                     score_mode=1 if args.score == "count" else 0, device=dev)
            print(json.dumps(out), flush=True)
    else:
        for d in args.d:
            for band in (args.band or [None]):
                kw = dict(model="banded", band=band) if band is not None else {}
                for row in phase_transition(ccs, n=2 ** args.n_log2, d=d, deltas=args.deltas,
                                            per_point=args.per_point, seed=args.seed, device=dev,
                                            **kw):
                    if band is not None:
                        row["band"] = band
                    print(json.dumps(row), flush=True)


if __name__ == "__main__":
    _main()

"""Phase transitions of Parallel-l0 on the GPU (Sec. 5.1, Sec. 5.6).

The protocol of Sec. 5.1: for each delta = m/n, start at rho = k/m = 0.01,
decode a few random problems per point and raise rho by 0.01 while at least
one of them is recovered; fit a logistic curve to the recovery data and
report its 50 % point rho*(delta).  Here every point's problems go to the
GPU as one batched decode (the points of a delta are sent in chunks; the
stopping rule is applied to the collected data, so the data equal those of
the sequential protocol).  Recovery is the outcome CONVERGED with x_hat == x
(on the default gauss-grid values every sum is exact, so this is the
paper's 1e-6 tolerance with nothing to round).

Banded signals (Sec. 5.6): the same sweep with a fraction `band` of the
support sharing one value.
"""
from __future__ import annotations

import math

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
                y = ccs.measure(ptr, cols, torch.from_numpy(p.x).to(device), m, d)
                probs.append(p)
                items.append((csc, ptr, cols, y))
        outs = ccs.decode_batch(items)
        for ci, rho in enumerate(rhos):
            ok = 0
            for t in range(per_point):
                q = ci * per_point + t
                rec = outs[q].status == ccs.CONVERGED and bool(
                    (outs[q].x_hat.cpu().numpy() == probs[q].x).all())
                data.append((rho, rec))
                ok += rec
            if ok == 0:  # the protocol stops at the first point with no recovery
                done = True
                break
        step += len(rhos)
        del items, outs
    rho_arr = np.array([r for r, _ in data])
    suc = np.array([s for _, s in data], dtype=np.float64)
    c, b = logistic_fit(rho_arr, suc)
    return {"delta": delta, "m": m, "rho_star": c, "slope": b, "points": len(data) // per_point,
            "recovered": int(suc.sum()), "decodes": int(suc.size)}


def phase_transition(ccs, n: int = 2 ** 18, d: int = 7, deltas=None, per_point: int = 10,
                     seed: int = 20151508, model: str = "gauss-grid", band: float = 0.0,
                     device="cuda") -> list[dict]:
    """rho*(delta) for each delta (default: the paper's 24 values)."""
    deltas = paper_deltas() if deltas is None else list(deltas)
    return [sweep_delta(ccs, n, d, dl, per_point=per_point, seed=seed + 101 * i, model=model,
                        band=band, device=device) for i, dl in enumerate(deltas)]

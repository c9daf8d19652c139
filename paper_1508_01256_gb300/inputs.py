"""Seeded synthetic inputs for expander l0-decoding.

This module only draws random inputs: it holds none of the decoder's
arithmetic (no y = A x, no score, no residual).  The CUDA path and the CPU
oracle both take their inputs from here.

Shapes follow the experiments of Sec. 5 of the paper (Mendoza-Smith & Tanner,
"Expander l0-decoding"): nonzeros of x drawn from N(0, 1) on a uniformly
random support, delta = m/n, rho = k/m, d ones per column.  The expander
matrix itself is produced by the library's ``ccs_make_expander`` from a
64-bit seed; this module only chooses that seed.

Value models (all host-side, numpy's PCG64 + ziggurat normal sampler):

``gauss-grid`` (default)
    N(0,1) rounded to the grid 2^-32 (values with |g| >= 8 or rounding to 0
    are redrawn).  Every sum of at most 2^17 such values is exact in
    binary64, so exact equality of residual entries means equality of the
    real sums and recovery depends on the combinatorics alone.
``gauss-raw``
    literal binary64 N(0,1) draws.
``pm1``
    iid Rademacher signs, a non-dissociated signal (Sec. 4.3, 5.5).
``banded``
    a fraction ``band`` of the support shares one N(0,1) value, the rest are
    independent (the almost-dissociated signals of Sec. 5.5).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 20151508
VALUE_MODELS = ("gauss-grid", "gauss-raw", "pm1", "banded")
_GRID = 2.0 ** -32


def round_half_up(v: float) -> int:
    return int(math.floor(v + 0.5))


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed & (2**63 - 1), stream])))


def expander_seed(seed: int) -> int:
    """64-bit seed handed to ccs_make_expander for problem ``seed``."""
    return int(_rng(seed, 1).integers(0, 2**63 - 1, dtype=np.int64)) * 2 + 1


def support(n: int, k: int, seed: int) -> np.ndarray:
    """Uniform random k-subset of [0, n), ascending (int64)."""
    if k < 0 or k > n:
        raise ValueError(f"k={k} outside [0, n={n}]")
    rng = _rng(seed, 2)
    return np.sort(rng.choice(n, size=k, replace=False)).astype(np.int64)


def values(k: int, seed: int, model: str = "gauss-grid", band: float = 0.0) -> np.ndarray:
    rng = _rng(seed, 3)
    if model == "gauss-raw":
        v = rng.standard_normal(k)
        while np.any(v == 0.0):  # a zero would shrink the support
            z = v == 0.0
            v[z] = rng.standard_normal(int(z.sum()))
        return v
    if model in ("gauss-grid", "banded"):
        v = np.empty(k, dtype=np.float64)
        filled = 0
        while filled < k:
            g = rng.standard_normal(k - filled)
            q = np.rint(g / _GRID) * _GRID
            ok = (np.abs(g) < 8.0) & (q != 0.0)
            q = q[ok]
            v[filled:filled + q.size] = q
            filled += q.size
        if model == "banded" and k > 0:
            nb = round_half_up(band * k)
            if nb > 0:
                common = v[0]
                pick = rng.choice(k, size=nb, replace=False)
                v[pick] = common
        return v
    if model == "pm1":
        return np.where(rng.integers(0, 2, size=k) == 1, 1.0, -1.0)
    raise ValueError(f"unknown value model {model!r}")


@dataclasses.dataclass
class Problem:
    """One synthetic instance: sizes, expander seed and the signal x, kept as
    its support ``idx`` (ascending) and values ``val``; ``x`` is the dense
    vector, built on first use."""
    n: int
    m: int
    d: int
    k: int
    seed: int
    model: str
    a_seed: int
    idx: np.ndarray  # int64[k]
    val: np.ndarray  # float64[k]
    _x: np.ndarray | None = dataclasses.field(default=None, repr=False, compare=False)

    @property
    def x(self) -> np.ndarray:
        """Dense float64[n] signal."""
        if self._x is None:
            x = np.zeros(self.n, dtype=np.float64)
            x[self.idx] = self.val
            self._x = x
        return self._x

    @property
    def support(self) -> np.ndarray:
        return self.idx

    def x_device(self, device="cuda"):
        """The dense signal as a device tensor, scattered on the device from
        the support and values (no dense host copy)."""
        import torch
        x = torch.zeros(self.n, dtype=torch.float64, device=device)
        x[torch.from_numpy(self.idx).to(device)] = torch.from_numpy(self.val).to(device)
        return x


def make_problem(n: int, m: int, d: int, k: int, seed: int,
                 model: str = "gauss-grid", band: float = 0.0) -> Problem:
    if not (1 <= d <= m) or n < 1:
        raise ValueError(f"bad sizes n={n} m={m} d={d}")
    s = support(n, k, seed)
    v = values(k, seed, model, band)
    return Problem(n, m, d, k, seed, model, expander_seed(seed), s, v)


# ---------------------------------------------------------------------------
# Workloads shaped like the paper's experiments
# ---------------------------------------------------------------------------

def plain_small(seed: int = BASE_SEED, model: str = "gauss-grid") -> Problem:
    """n=4096, m=410, k=41, d=7 (delta ~ 0.1, rho = 0.1)."""
    return make_problem(4096, 410, 7, 41, seed, model)


def plain_at_scale(seed: int = BASE_SEED, model: str = "gauss-grid") -> Problem:
    """n=2^20, m=2^17, k=round(0.2 m)=26214, d=7 (Sec. 5.3/5.4 shapes)."""
    m = 2 ** 17
    return make_problem(2 ** 20, m, 7, round_half_up(0.2 * m), seed, model)


EXTREME_RHOS = (0.05, 0.10, 0.15, 0.20, 0.25, 0.30)


def extreme_undersampling(rho: float, d: int = 9, seed: int = BASE_SEED,
                          model: str = "gauss-grid", log2n: int = 24) -> Problem:
    """delta = m/n ~ 10^-3 (Sec. 5.5, Table 3 shape): n=2^24, m=16777."""
    n = 2 ** log2n
    m = round_half_up(n * 1e-3)
    return make_problem(n, m, d, round_half_up(rho * m), seed, model)


BATCH_DELTAS = (0.01, 0.05, 0.1, 0.3)
BATCH_RHOS = (0.05, 0.1, 0.2)
BATCH_DS = (5, 7, 9, 11)


def batch_shapes(count: int = 512, seed: int = BASE_SEED, log2n_lo: float = 12.0,
                 log2n_hi: float = 20.0, ds=BATCH_DS):
    """(n, m, d, k) of a mixed batch: n log-uniform in [2^lo, 2^hi], delta,
    rho and d drawn uniformly from the sets above."""
    rng = _rng(seed, 7)
    out = []
    for _ in range(count):
        u = rng.uniform(log2n_lo, log2n_hi)
        n = int(round(2.0 ** u))
        delta = float(rng.choice(BATCH_DELTAS))
        rho = float(rng.choice(BATCH_RHOS))
        d = int(rng.choice(ds))
        m = max(d, round_half_up(delta * n))
        k = round_half_up(rho * m)
        out.append((n, m, d, k))
    return out


def batch_problems(count: int = 512, seed: int = BASE_SEED, model: str = "gauss-grid",
                   **kw) -> list[Problem]:
    shapes = batch_shapes(count, seed, **kw)
    return [make_problem(n, m, d, k, seed * 1000003 + p, model)
            for p, (n, m, d, k) in enumerate(shapes)]


def poisson_arrivals(count: int, rate_per_s: float, seed: int = BASE_SEED) -> np.ndarray:
    """Arrival times (s) of a Poisson process with the given rate."""
    rng = _rng(seed, 9)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))

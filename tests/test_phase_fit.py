"""The logistic fit of the phase-transition driver (Sec. 5.1), on synthetic
recovery data with a known 50 % point."""
import math

import numpy as np

from paper_1508_01256_gb300 import phase


def test_paper_deltas():
    ds = phase.paper_deltas()
    assert len(ds) == 24
    assert np.allclose(ds[:4], [0.02, 0.04, 0.06, 0.08])
    assert math.isclose(ds[4], 0.1) and math.isclose(ds[-1], 0.1 + 89 / 1900 * 19)


def test_logistic_fit_recovers_known_transition():
    rng = np.random.default_rng(3)
    rho = np.repeat(np.arange(0.01, 0.61, 0.01), 40)
    c0, b0 = 0.32, 45.0
    p = 1.0 / (1.0 + np.exp(b0 * (rho - c0)))
    success = rng.random(rho.size) < p
    c, b = phase.logistic_fit(rho, success)
    assert abs(c - c0) < 0.01 and abs(b - b0) / b0 < 0.2


def test_logistic_fit_without_a_transition():
    c, _ = phase.logistic_fit(np.array([0.1, 0.2]), np.array([1.0, 1.0]))
    assert math.isnan(c)

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


def test_separated_data_report_a_bracket():
    """Every problem recovered up to rho = 0.34, none from 0.35: the logistic
    likelihood has no maximum, so the transition is the bracket, not a
    fitted number (and two different cliffs give different answers)."""
    rho = np.repeat(np.arange(0.01, 0.355, 0.01), 5)
    ok = rho < 0.345
    tr = phase.transition(rho, ok)
    assert tr["method"] == "bracket"
    assert np.allclose(tr["bracket"], [0.34, 0.35]) and math.isclose(tr["rho_star"], 0.345)
    rho2 = np.repeat(np.arange(0.01, 0.235, 0.01), 5)
    tr2 = phase.transition(rho2, rho2 < 0.225)
    assert np.allclose(tr2["bracket"], [0.22, 0.23])


def test_successes_and_failures_meeting_at_one_rho():
    rho = np.array([0.1, 0.1, 0.2, 0.2, 0.3, 0.3])
    ok = np.array([1, 1, 1, 0, 0, 0], dtype=bool)
    tr = phase.transition(rho, ok)
    assert tr["method"] == "bracket" and tr["bracket"] == [0.2, 0.2]


def test_overlapping_data_take_the_logistic_fit():
    rho = np.array([0.1, 0.1, 0.2, 0.2, 0.3, 0.3, 0.4, 0.4])
    ok = np.array([1, 1, 1, 0, 1, 0, 0, 0], dtype=bool)
    tr = phase.transition(rho, ok)
    assert tr["method"] == "logistic" and 0.2 < tr["rho_star"] < 0.3
    assert tr["slope"] > 0


def test_transition_without_data_on_both_sides():
    assert phase.transition([0.1, 0.2], [True, True])["method"] == "none"

"""The seeded input recipes match the workloads they stand for (the
synthetic instances of Sec. 5: uniform supports, N(0,1) nonzeros, delta =
m/n, rho = k/m, d ones per column) and are reproducible from their seeds.
Both the CUDA path and the oracle take their inputs from this module."""
import math

import numpy as np
import pytest

from paper_1508_01256_gb300 import inputs


def test_round_half_up():
    assert [inputs.round_half_up(v) for v in (0.5, 1.5, 2.49, 26214.4)] == [1, 2, 2, 26214]


def test_support_is_a_sorted_k_subset_and_uniform():
    for n, k in ((1, 0), (1, 1), (50, 50), (1000, 37)):
        s = inputs.support(n, k, 3)
        assert s.size == k and np.all(np.diff(s) > 0) and (k == 0 or (s[0] >= 0 and s[-1] < n))
    with pytest.raises(ValueError):
        inputs.support(5, 6, 1)
    # every position of [0, 10) is in a 3-subset with probability 3/10
    counts = np.zeros(10)
    trials = 4000
    for seed in range(trials):
        counts[inputs.support(10, 3, seed)] += 1
    expected = trials * 3 / 10
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    assert chi2 < 27.9  # chi^2 with 9 degrees of freedom at p = 0.001


def test_make_problem_places_k_values_on_the_support():
    p = inputs.make_problem(5000, 500, 7, 123, 42)
    assert p.x.shape == (5000,) and p.x.dtype == np.float64
    assert np.array_equal(p.support, inputs.support(5000, 123, 42))
    assert np.array_equal(p.x[p.support], inputs.values(123, 42))
    assert p.a_seed % 2 == 1 and 0 < p.a_seed < 2 ** 64
    q = inputs.make_problem(5000, 500, 7, 123, 42)
    assert np.array_equal(p.x, q.x) and p.a_seed == q.a_seed  # reproducible
    r = inputs.make_problem(5000, 500, 7, 123, 43)
    assert not np.array_equal(p.x, r.x) and p.a_seed != r.a_seed
    with pytest.raises(ValueError):
        inputs.make_problem(10, 5, 6, 1, 1)  # d > m


def test_named_workloads():
    s = inputs.plain_small()
    assert (s.n, s.m, s.d, s.k) == (4096, 410, 7, 41)
    a = inputs.plain_at_scale()
    assert (a.n, a.m, a.d, a.k) == (2 ** 20, 2 ** 17, 7, 26214)
    for rho in inputs.EXTREME_RHOS:
        e = inputs.extreme_undersampling(rho, log2n=20)
        assert e.m == inputs.round_half_up(2 ** 20 * 1e-3) and e.k == inputs.round_half_up(rho * e.m)
    assert inputs.round_half_up(2 ** 24 * 1e-3) == 16777  # the n = 2^24 shape


def test_batch_shapes_follow_the_mix():
    shapes = inputs.batch_shapes(2000, seed=11)
    deltas, rhos, ds = [], [], []
    for n, m, d, k in shapes:
        assert 2 ** 12 <= n <= 2 ** 20 and d in inputs.BATCH_DS
        cand = [dl for dl in inputs.BATCH_DELTAS if m == max(d, inputs.round_half_up(dl * n))]
        assert cand, (n, m, d)
        rc = [r for r in inputs.BATCH_RHOS if k == inputs.round_half_up(r * m)]
        assert rc, (m, k)
        deltas.append(cand[0])
        rhos.append(rc[0])
        ds.append(d)
    # each choice is drawn uniformly: every value takes its share, within 5 sigma
    for vals, choices in ((deltas, inputs.BATCH_DELTAS), (rhos, inputs.BATCH_RHOS),
                          (ds, inputs.BATCH_DS)):
        p = 1.0 / len(choices)
        for c in choices:
            share = sum(v == c for v in vals)
            assert abs(share - p * len(vals)) < 5 * math.sqrt(len(vals) * p * (1 - p)) + 1, c
    # log2 n is uniform on [12, 20]: its mean is 16
    assert abs(np.mean([math.log2(n) for n, _, _, _ in shapes]) - 16.0) < 0.25
    # the serving mix reaches 2^22 with d in {7, 9}
    serve = inputs.batch_shapes(500, seed=5, log2n_hi=22.0, ds=(7, 9))
    assert max(n for n, _, _, _ in serve) > 2 ** 20 and {d for _, _, d, _ in serve} == {7, 9}


def test_poisson_arrivals():
    t = inputs.poisson_arrivals(20000, 1000.0, seed=4)
    assert np.all(np.diff(t) > 0) and t[0] > 0
    gaps = np.diff(np.concatenate(([0.0], t)))
    assert abs(gaps.mean() - 1e-3) < 5e-5 and abs(gaps.std() - 1e-3) < 5e-5  # exponential

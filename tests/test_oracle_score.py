"""Pins for the oracle's score step (selection rule Eq. (15), Alg. 8).

The oracle computes the l0 decrease as c_omega - c_0 from the d gathered
values only.  Here it is checked against the literal definition
||r||_0 - ||r - omega a_j||_0 evaluated on the whole m-vector for every
candidate omega.
"""
import numpy as np
import pytest


def _l0(v):
    return int(np.count_nonzero(v))


def _literal_best(A, j, r, alpha, count_mode):
    """Evaluate every candidate omega (each nonzero value of r on N(j)) by the
    definition; return (accepted, omega, score) with ties to the smallest
    omega (reading R1)."""
    m = r.size
    a_j = np.zeros(m)
    a_j[A[j]] = 1.0
    cands = sorted(set(float(v) for v in r[A[j]] if v != 0.0))
    best = None
    for w in cands:
        if count_mode:
            s = int(np.sum(r[A[j]] == w))
        else:
            s = _l0(r) - _l0(r - w * a_j)
        if best is None or s > best[1]:
            best = (w, s)
    if best is None:
        return False, None, None
    return best[1] >= alpha, best[0], best[1]


def _random_residual(rng, m, nvals):
    pool = np.rint(rng.standard_normal(nvals) * 2 ** 20) / 2 ** 20
    r = rng.choice(np.concatenate([pool, [0.0, 0.0, -0.0]]), size=m)
    return r


@pytest.mark.parametrize("d", [1, 2, 3, 5, 7, 9, 11, 16])
@pytest.mark.parametrize("count_mode", [False, True])
def test_score_matches_literal_definition(orc, d, count_mode):
    rng = np.random.default_rng(d * 7 + count_mode)
    n, m = 400, 40
    A = orc.make_expander(n, m, d, 77 + d)
    mode = orc.SCORE_COUNT if count_mode else orc.SCORE_L0_DECREASE
    for trial in range(6):
        r = _random_residual(rng, m, nvals=2 + trial * 2)
        for alpha in (2, 3, max(2, d)):
            acc, om, sc = orc.score_all(A, r, alpha, mode)
            for j in range(n):
                a, w, s = _literal_best(A, j, r, alpha, count_mode)
                assert acc[j] == a, (j, a, w, s)
                if w is not None:
                    # chosen omega maximises the literal score, smallest first
                    assert om[j] == w and sc[j] == s


def test_score_hand_built_columns(orc):
    rows = np.arange(7, dtype=np.int32)
    # all zero: nothing to choose
    acc, om, sc, ct = orc.score_column(rows, np.zeros(7))
    assert not acc and ct == 0
    # all equal nonzero: score d
    acc, om, sc, ct = orc.score_column(rows, np.full(7, 0.25))
    assert acc and om == 0.25 and sc == 7 and ct == 7
    # tie between two values: the smaller one wins
    r = np.array([3.0, 3.0, -1.0, -1.0, 5.0, 6.0, 7.0])
    acc, om, sc, ct = orc.score_column(rows, r)
    assert acc and om == -1.0 and sc == 2
    # zeros lower the l0 decrease but not the match count
    r = np.array([2.0, 2.0, 0.0, 0.0, -0.0, 6.0, 7.0])
    acc, om, sc, ct = orc.score_column(rows, r, alpha=2)
    assert not acc and om == 2.0 and sc == -1 and ct == 2
    acc, om, sc, ct = orc.score_column(rows, r, alpha=2, score_mode=orc.SCORE_COUNT)
    assert acc and sc == 2
    # all distinct: best count 1 -> never accepted since alpha >= 2
    acc, om, sc, ct = orc.score_column(rows, np.arange(1.0, 8.0))
    assert not acc and ct == 1 and om == 1.0
    # -0.0 is zero, +0.0 and -0.0 are the same value
    r = np.array([-0.0, 0.0, 4.0, 4.0, 4.0, 1.0, 1.0])
    acc, om, sc, ct = orc.score_column(rows, r)
    assert not acc and om == 4.0 and sc == 1 and ct == 3


@pytest.mark.parametrize("d", [1, 3, 5, 7, 9, 16])
@pytest.mark.parametrize("count_mode", [False, True])
def test_shifted_score_matches_literal_definition(orc, d, count_mode):
    """Shifted variant (Sec. 4.3.1): the candidate is r at the pos-th row of
    N(j) (rows ascending); its score is checked against the literal
    ||r||_0 - ||r - omega a_j||_0 on the whole vector (or the match count),
    and a zero candidate is never accepted."""
    rng = np.random.default_rng(100 + d * 7 + count_mode)
    n, m = 300, 40
    A = orc.make_expander(n, m, d, 55 + d)
    assert np.all(np.diff(A, axis=1) > 0)  # rows ascending within a column
    mode = orc.SCORE_COUNT if count_mode else orc.SCORE_L0_DECREASE
    for trial in range(5):
        r = _random_residual(rng, m, nvals=2 + trial)
        for pos in range(d):
            for alpha in (2, max(2, d)):
                acc, om, sc = orc.score_all(A, r, alpha, mode, shift_pos=pos)
                for j in range(n):
                    w = float(r[A[j][pos]])
                    a_j = np.zeros(m)
                    a_j[A[j]] = 1.0
                    if w == 0.0:
                        assert not acc[j]
                        continue
                    lit = int(np.sum(r[A[j]] == w)) if count_mode else \
                        _l0(r) - _l0(r - w * a_j)
                    assert om[j] == w and sc[j] == lit
                    assert bool(acc[j]) == (lit >= alpha)
                    a1, w1, s1, _ = orc.score_column_shifted(A[j], r, pos, alpha, mode)
                    assert (a1, w1, s1) == (bool(acc[j]), w, lit)

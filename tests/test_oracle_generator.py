"""Pins for the oracle's expander generator, transpose and y = A x.

The generator follows the Sec. 1.1 footnote of the paper (columns drawn iid,
each uniform over the C(m, d) supports of size d); the transpose gives N(i)
for each row; the measurement is y = A x with the row-sum rule (ascending
column order, from +0.0).
"""
import itertools
import os

import numpy as np
import pytest

from paper_1508_01256_gb300 import inputs

import rejection_seeds

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_hex(name):
    vals = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                vals.append(int(line, 16))
    return vals


def test_splitmix64_published_vector(orc):
    assert orc.splitmix64(0, 3) == _golden_hex("splitmix64_seed0.txt")


@pytest.mark.parametrize("n,m,d", [(1, 1, 1), (7, 7, 7), (300, 40, 5), (2000, 410, 7),
                                   (500, 17, 16), (64, 100000, 3)])
def test_expander_columns_distinct_sorted(orc, n, m, d):
    A = orc.make_expander(n, m, d, 12345)
    assert A.shape == (n, d)
    assert A.min() >= 0 and A.max() < m
    assert np.all(np.diff(A, axis=1) > 0)  # ascending => distinct


def test_expander_deterministic_and_seeded(orc):
    a = orc.make_expander(1000, 97, 7, 5)
    b = orc.make_expander(1000, 97, 7, 5)
    c = orc.make_expander(1000, 97, 7, 6)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)


def test_expander_rejects_bad_sizes(orc):
    with pytest.raises(ValueError):
        orc.make_expander(10, 3, 4, 1)  # d > m: no d distinct rows exist


def test_expander_supports_uniform(orc):
    """Each column's support is uniform over the C(m, d) subsets."""
    from scipy.stats import chisquare
    m, d, n = 7, 3, 70000
    A = orc.make_expander(n, m, d, 99)
    subsets = {s: i for i, s in enumerate(itertools.combinations(range(m), d))}
    idx = np.array([subsets[tuple(r)] for r in A.tolist()])
    counts = np.bincount(idx, minlength=len(subsets))
    assert chisquare(counts).pvalue > 1e-4


def test_expander_row_degrees(orc):
    """Row degrees: mean d n / m, and the row counts are uniform over rows."""
    from scipy.stats import chisquare
    n, m, d = 60000, 97, 5
    A = orc.make_expander(n, m, d, 3)
    deg = np.bincount(A.ravel(), minlength=m)
    assert deg.sum() == n * d
    assert chisquare(deg).pvalue > 1e-4
    # draws within a column: position 0 is the minimum of d uniform distinct
    # rows, so its mean is (m + 1)/(d + 1) - 1 for 0-based rows
    assert abs(A[:, 0].mean() - ((m + 1) / (d + 1) - 1)) < 0.3


def test_transpose_round_trip(orc):
    n, m, d = 3000, 211, 7
    A = orc.make_expander(n, m, d, 8)
    ptr, cols = orc.transpose(A, m)
    assert ptr[0] == 0 and ptr[-1] == n * d
    assert np.all(np.diff(ptr) >= 0)
    back = [[] for _ in range(n)]
    for i in range(m):
        seg = cols[ptr[i]:ptr[i + 1]]
        assert np.all(np.diff(seg) > 0)  # each row's columns ascending
        for j in seg:
            back[j].append(i)
    assert np.array_equal(np.array(back, dtype=np.int32), A)


def test_measure_exact_on_grid(orc):
    """On the 2^-32 grid every sum is exact, so y equals the integer sum."""
    p = inputs.make_problem(5000, 600, 7, 300, 11)
    A = orc.make_expander(p.n, p.m, p.d, p.a_seed)
    y = orc.measure(A, p.m, p.x)
    xi = [int(v) for v in np.rint(p.x * 2.0 ** 32)]
    acc = [0] * p.m
    for j in np.nonzero(p.x)[0]:
        for i in A[j]:
            acc[i] += xi[j]
    assert np.array_equal(y, np.array([a * 2.0 ** -32 for a in acc]))


def test_row_sum_is_ascending_sequential(orc):
    """The row sum adds in ascending column order (reading of the residual
    step of Alg. 2): with x = (1e16, 1, -1e16) on one row, the ascending sum
    is (1e16 + 1) - 1e16 = 0 in binary64 (1e16 + 1 rounds to 1e16), while
    any order that adds 1 last would give 1."""
    A = np.array([[0], [0], [0]], dtype=np.int32)  # n=3, m=1, d=1
    x = np.array([1e16, 1.0, -1e16])
    y = orc.measure(A, 1, x)
    assert y[0] == 0.0
    r = orc.residual(A, 1, np.array([5.0]), x)
    assert r[0] == 5.0
    # two rows whose sums tell ascending from descending order apart:
    # row 0 holds (1, 1e16, -1e16): ascending (1 + 1e16) - 1e16 = 0, while
    # descending (-1e16 + 1e16) + 1 = 1; row 1 holds (1e16, -1e16, 1):
    # ascending 1, descending (1 - 1e16) + 1e16 = 0
    A2 = np.array([[0], [0], [0], [1], [1], [1]], dtype=np.int32)
    x2 = np.array([1.0, 1e16, -1e16, 1e16, -1e16, 1.0])
    assert orc.measure(A2, 2, x2).tolist() == [0.0, 1.0]
    assert orc.residual(A2, 2, np.array([3.0, 3.0]), x2).tolist() == [3.0, 2.0]
    # skip zeros and start from +0.0: an all-zero row gives +0.0
    y0 = orc.measure(A, 1, np.array([0.0, -0.0, 0.0]))
    assert y0[0] == 0.0 and not np.signbit(y0[0])


def test_values_models():
    v = inputs.values(10000, 5, "gauss-grid")
    assert np.all(v != 0) and np.all(np.abs(v) < 8)
    assert np.array_equal(v, np.rint(v * 2.0 ** 32) * 2.0 ** -32)
    assert abs(v.mean()) < 0.05 and abs(v.std() - 1) < 0.05
    pm = inputs.values(1000, 5, "pm1")
    assert set(np.unique(pm)) == {-1.0, 1.0}
    b = inputs.values(1000, 5, "banded", band=0.5)
    assert np.max(np.unique(b, return_counts=True)[1]) >= 500


def test_bounded_draw_rejection_branch(orc):
    """Lemire's bounded draw maps x to floor(x m / 2^64) but first rejects x
    when the low word x m mod 2^64 is below (2^64 - m) mod m, which makes every
    row exactly equally likely.  The branch fires with probability about
    m / 2^64, so random tests never reach it: the seeds of rejection_seeds
    make column 0 first draw such an x (m = 6).  The row must come from the
    first draw that is not rejected."""
    M64, m = rejection_seeds.M64, rejection_seeds.M
    threshold = (M64 - m) % m
    differs = []
    for x0, seed in rejection_seeds.rejected_first_draws():
        assert (x0 * m) % M64 < threshold
        draws = orc.splitmix64((seed + rejection_seeds.COLUMN_STEP) % M64, 8)
        assert draws[0] == x0
        accepted = next(x for x in draws[1:] if (x * m) % M64 >= threshold)
        row = (accepted * m) >> 64
        assert orc.make_expander(1, m, 1, seed)[0, 0] == row
        differs.append(row != (x0 * m) >> 64)
    assert any(differs)  # the rejected draw would have given another row

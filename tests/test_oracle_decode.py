"""Pins for the oracle's Parallel-l0 (Alg. 2) and Serial-l0 (Alg. 1).

The theorem-regime cases use the point-line incidence matrix of the affine
plane AG(2, q) (q prime): its q^2 + q lines are the columns, its q^2 points
the rows, d = q, and two columns share at most one row.  For those graphs the
expansion parameter eps of Def. 2 is found by brute force over all column
sets of size <= k, and Theorem 1 (with Lemmas 1-6 and Eq. (37)) then fixes
what the decoder must do: accept only exact values x_j at the right j,
shrink the support of x - x_hat by the factor of Eq. (37) every iteration,
and end with x_hat = x, which brute force over all supports of size <= k
confirms to be the unique sparsest solution.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_1508_01256_gb300 import inputs


def affine_plane(q):
    lines = []
    for s in range(q):
        for c in range(q):
            lines.append(sorted(a * q + (s * a + c) % q for a in range(q)))
    for c in range(q):
        lines.append(sorted(c * q + b for b in range(q)))
    return np.array(lines, dtype=np.int32)


def eps_star(A, m, k):
    """max over 1 <= |S| <= k of 1 - |N(S)|/(d|S|): the graph is a
    (k, eps, d)-expander exactly for eps > eps_star (Def. 2)."""
    n, d = A.shape
    nbrs = [frozenset(map(int, r)) for r in A]
    worst = Fraction(0)
    for size in range(1, k + 1):
        for S in itertools.combinations(range(n), size):
            u = frozenset().union(*(nbrs[j] for j in S))
            worst = max(worst, 1 - Fraction(len(u), d * size))
    return worst


def dissociated(vals):
    ints = [int(v) for v in np.rint(np.asarray(vals) * 2.0 ** 32)]
    sums = set()
    for size in range(len(ints) + 1):
        for T in itertools.combinations(ints, size):
            sums.add(sum(T))
    return len(sums) == 2 ** len(ints)


def dense(A, m):
    n, _ = A.shape
    M = np.zeros((m, n))
    for j in range(n):
        M[A[j], j] = 1.0
    return M


def unique_sparsest(M, y, k):
    """All supports of size <= k whose least-squares fit reproduces y."""
    m, n = M.shape
    fits = []
    for size in range(0, k + 1):
        combos = np.array(list(itertools.combinations(range(n), size)), dtype=np.int64)
        if size == 0:
            if np.all(y == 0):
                fits.append(())
            continue
        for chunk in np.array_split(combos, max(1, len(combos) // 4000)):
            As = M[:, chunk].transpose(1, 0, 2)          # (N, m, size)
            c = np.linalg.pinv(As) @ y                   # (N, size)
            res = np.linalg.norm(As @ c[:, :, None] - y[None, :, None], axis=(1, 2))
            for t in np.nonzero(res < 1e-9)[0]:
                fits.append(tuple(chunk[t]))
    return fits


def _theorem_cases():
    cases = []
    for q, k in ((5, 3), (7, 3), (7, 4)):
        for seed in range(3):
            cases.append((q, k, seed))
    return cases


@pytest.mark.parametrize("q,k,seed", _theorem_cases())
def test_theorem_regime(orc, q, k, seed):
    rng = np.random.default_rng(1000 * q + 10 * k + seed)
    A = affine_plane(q)
    # random relabelling of rows keeps the incidence structure
    perm = rng.permutation(q * q).astype(np.int32)
    A = np.sort(perm[A], axis=1).astype(np.int32)
    n, d = A.shape
    m = q * q
    es = eps_star(A, m, k)
    assert es < Fraction(1, 4)
    alpha = math.ceil((1 - 2 * es) * d)  # integer threshold of (1-2eps)d, eps -> eps*+
    eps = float(es) + 1e-9
    ratio = 2 * eps * d / (1 + math.floor(2 * eps * d))
    ell_star = 0
    while k * ratio ** ell_star >= 1:
        ell_star += 1

    x = np.zeros(n)
    supp = np.sort(rng.choice(n, size=k, replace=False))
    x[supp] = inputs.values(k, seed + 17 * q + k, "gauss-grid")
    assert dissociated(x[supp])
    y = orc.measure(A, m, x)

    res = orc.parallel_l0(A, m, y, alpha=alpha, max_iter=50, trace=True)
    assert res["status"] == orc.CONVERGED
    assert np.array_equal(res["x_hat"], x)
    assert res["iterations"] <= ell_star
    h = res["r0_hist"]
    assert np.all(np.diff(h) < 0)  # strict contraction of ||r||_0
    # replay the trace: every accepted pair is (j, x_j) with j still wrong
    xh = np.zeros(n)
    for it, idx, om in res["trace"]:
        S = set(np.nonzero(x - xh)[0])
        assert len(idx) > 0
        for j, w in zip(idx, om):
            assert j in S and xh[j] == 0.0 and w == x[j]
        xh[idx] += om
        S_next = set(np.nonzero(x - xh)[0])
        assert len(S_next) <= ratio * len(S) + 1e-12
    # brute force: x is the only support of size <= k that explains y
    fits = unique_sparsest(dense(A, m), y, k)
    assert fits == [tuple(supp)]
    # Serial-l0 (Alg. 1) also recovers x
    ser = orc.serial_l0(A, m, y, alpha=alpha, max_iter=50)
    assert ser["status"] == orc.CONVERGED and np.array_equal(ser["x_hat"], x)
    assert ser["iterations"] <= res["iterations"]
    # the shifted variants (Sec. 4.3.1) recover x too (their theorem: same
    # graphs, alpha = (1 - 2 eps) d); every pair they accept is (j, x_j)
    shp = orc.parallel_l0(A, m, y, alpha=alpha, max_iter=50 * d, trace=True, shifted=True)
    assert shp["status"] == orc.CONVERGED and np.array_equal(shp["x_hat"], x)
    xh = np.zeros(n)
    for it, idx, om in shp["trace"]:
        for j, w in zip(idx, om):
            assert xh[j] == 0.0 and w == x[j]
        xh[idx] += om
    shs = orc.serial_l0(A, m, y, alpha=alpha, max_iter=50 * d, shifted=True)
    assert shs["status"] == orc.CONVERGED and np.array_equal(shs["x_hat"], x)


def test_k0_converges_immediately(orc):
    A = orc.make_expander(300, 40, 5, 1)
    res = orc.parallel_l0(A, 40, np.zeros(40))
    assert res["status"] == orc.CONVERGED and res["iterations"] == 0
    assert np.all(res["x_hat"] == 0) and list(res["r0_hist"]) == [0]


@pytest.mark.parametrize("seed", range(8))
def test_k1_first_iteration_predicted(orc, seed):
    """k = 1: all d rows of the support column j0 hold x_j0 (score d); any
    other column with overlap o sees x_j0 o times and zero d - o times, so its
    l0 decrease is 2o - d.  The first accepted set is therefore exactly
    {j0} and the columns with 2o - d >= alpha; when that set is {j0} the
    decode ends after one iteration with x_hat = x."""
    n, m, d = 500, 60, 7
    A = orc.make_expander(n, m, d, 40 + seed)
    j0 = seed * 37 % n
    ov = np.array([len(set(A[j]) & set(A[j0])) for j in range(n)])
    predicted = sorted(set([j0]) | set(np.nonzero(2 * ov - d >= 2)[0].tolist()))
    x = np.zeros(n)
    x[j0] = inputs.values(1, seed, "gauss-grid")[0]
    y = orc.measure(A, m, x)
    res = orc.parallel_l0(A, m, y, trace=True)
    it0, idx, om = res["trace"][0]
    assert list(idx) == predicted and np.all(om == x[j0])
    if predicted == [j0]:
        assert res["status"] == orc.CONVERGED and res["iterations"] == 1
        assert np.array_equal(res["x_hat"], x)


def test_disjoint_neighbourhoods_one_iteration(orc):
    n, m, d = 40, 120, 3
    A = np.array([[3 * j + t for t in range(d)] for j in range(n)], dtype=np.int32)
    supp = [0, 1, 2, 3, 4]  # all neighbourhoods pairwise disjoint
    x = np.zeros(n)
    x[supp] = inputs.values(5, 3, "gauss-grid")
    y = orc.measure(A, m, x)
    res = orc.parallel_l0(A, m, y)
    assert res["status"] == orc.CONVERGED and res["iterations"] == 1
    assert np.array_equal(res["x_hat"], x)


def test_count_mode_spurious_acceptance(orc):
    """Column 1 shares two rows with the support column 0 and sees one zero:
    l0 decrease 2 - 1 = 1 < alpha, match count 2 >= alpha.  The two score
    readings of Eq. (15) vs Alg. 8 part here."""
    A = np.array([[0, 1, 2], [0, 1, 3], [2, 3, 4]], dtype=np.int32)
    y = np.array([0.5, 0.5, 0.5, 0.0, 0.0])
    l0 = orc.parallel_l0(A, 5, y, alpha=2)
    assert l0["status"] == orc.CONVERGED and l0["iterations"] == 1
    assert np.array_equal(l0["x_hat"], [0.5, 0.0, 0.0])
    cnt = orc.parallel_l0(A, 5, y, alpha=2, score_mode=orc.SCORE_COUNT,
                          max_iter=10, trace=True)
    assert list(cnt["trace"][0][1]) == [0, 1]
    assert cnt["status"] == orc.MAX_ITER  # it oscillates between two states


def test_stalled_when_nothing_qualifies(orc):
    A = np.array([[0, 1, 2], [2, 3, 4]], dtype=np.int32)
    y = np.array([1.0, 2.0, 3.0, 4.0, 5.0])  # all distinct, not in range of A
    res = orc.parallel_l0(A, 5, y)
    assert res["status"] == orc.STALLED and res["iterations"] == 0
    assert np.array_equal(res["r"], y)
    # Serial-l0 (Alg. 1) stops the same way: a sweep that accepts nothing
    ser = orc.serial_l0(A, 5, y, max_iter=50)
    assert ser["status"] == orc.STALLED and ser["iterations"] == 0
    assert np.array_equal(ser["r"], y) and not np.any(ser["x_hat"])
    # ... and after progress: column 0 explains rows 0-2 (value 1), the rest
    # is not in the range of A, so the second sweep accepts nothing
    y2 = np.array([1.0, 1.0, 1.0, 4.0, 5.0])
    ser = orc.serial_l0(A, 5, y2, max_iter=50)
    assert ser["status"] == orc.STALLED and ser["iterations"] == 1
    assert ser["x_hat"].tolist() == [1.0, 0.0]


def test_max_iter_zero(orc):
    A = np.array([[0, 1, 2]], dtype=np.int32)
    res = orc.parallel_l0(A, 3, np.array([1.0, 1.0, 1.0]), max_iter=0)
    assert res["status"] == orc.MAX_ITER and res["iterations"] == 0


@pytest.mark.parametrize("model", ["gauss-grid", "gauss-raw", "pm1"])
def test_convergence_invariant(orc, model):
    """CONVERGED <=> r == 0 <=> y == A x_hat under the row-sum rule; the
    returned r always equals y - A x_hat and r0 its l0 norm."""
    for s in range(5):
        p = inputs.make_problem(4096, 410, 7, 41 + 10 * s, 500 + s, model)
        A = orc.make_expander(p.n, p.m, p.d, p.a_seed)
        y = orc.measure(A, p.m, p.x)
        res = orc.parallel_l0(A, p.m, y)
        r_ref = y - dense(A, p.m) @ res["x_hat"] if model == "gauss-grid" else \
            orc.residual(A, p.m, y, res["x_hat"])
        assert np.array_equal(res["r"], r_ref)
        assert res["r0_final"] == np.count_nonzero(res["r"]) == res["r0_hist"][-1]
        conv = res["status"] == orc.CONVERGED
        assert conv == (res["r0_final"] == 0)
        if conv:
            assert np.array_equal(orc.measure(A, p.m, res["x_hat"]), y)


def test_small_workload_recovers(orc):
    """n=4096, m=410, k=41, d=7 (rho = 0.1, well under the phase transition
    of Sec. 5.1): every seeded instance is recovered exactly, in few
    iterations (Sec. 5.4 reports O(log k) iterations)."""
    for s in range(10):
        p = inputs.plain_small(seed=s)
        A = orc.make_expander(p.n, p.m, p.d, p.a_seed)
        y = orc.measure(A, p.m, p.x)
        res = orc.parallel_l0(A, p.m, y)
        assert res["status"] == orc.CONVERGED and np.array_equal(res["x_hat"], p.x)
        assert res["iterations"] <= math.ceil(math.log(41)) + 1


def test_shifted_k1_single_iteration(orc):
    """k = 1: at iteration 0 the shifted candidate of the support column is
    x_j itself (all its rows hold it), score d; a column sharing o rows with
    it has candidate x_j only when its first row is shared (score 2o - d in
    the l0 form) else 0, so with alpha = d only the support column is taken:
    one iteration, exact recovery."""
    A = orc.make_expander(2000, 300, 7, 9)
    x = np.zeros(2000)
    x[777] = 1.25
    y = orc.measure(A, 300, x)
    res = orc.parallel_l0(A, 300, y, alpha=7, shifted=True)
    assert res["status"] == orc.CONVERGED and res["iterations"] == 1
    assert np.array_equal(res["x_hat"], x)


def test_column_scales_grid_and_distribution(orc):
    """Reading R12: s_j on [1, 2), multiples of 2^-20, close to uniform, and
    a different sequence for another seed."""
    s = orc.column_scales(200000, 5)
    assert np.all((s >= 1.0) & (s < 2.0))
    k = (s - 1.0) * 2 ** 20
    assert np.array_equal(k, np.floor(k))
    assert abs(s.mean() - 1.5) < 0.003 and abs(s.std() - (1 / 12) ** 0.5) < 0.003
    hist = np.histogram(s, bins=16, range=(1.0, 2.0))[0]
    assert hist.min() > 0.9 * 200000 / 16
    assert not np.array_equal(s[:100], orc.column_scales(100, 6))


def test_measure_scaled_is_the_exact_sum(orc):
    """y = A diag(s) x on +/-1 and small-integer x equals the exact rational
    sum (integer arithmetic on the 2^-20 grid)."""
    n, m, d = 3000, 300, 7
    A = orc.make_expander(n, m, d, 3)
    s = orc.column_scales(n, 11)
    rng = np.random.default_rng(4)
    x = np.zeros(n)
    supp = rng.choice(n, 200, replace=False)
    x[supp] = rng.choice([-3.0, -1.0, 1.0, 2.0], 200)
    y = orc.measure_scaled(A, m, s, x)
    si = ((s - 1.0) * 2 ** 20).astype(np.int64) + 2 ** 20      # s_j * 2^20
    exact = np.zeros(m, dtype=np.int64)
    for j in supp:
        for i in A[j]:
            exact[i] += si[j] * int(x[j])
    assert np.array_equal(y * 2 ** 20, exact.astype(np.float64))


def test_measure_scaled_order_and_rounding(orc):
    """Each product s_j x_j is rounded once and the row adds them in
    ascending column order from +0.0 (readings R6, R12).  With s = 1, the
    rows (1, 1e16, -1e16) and (1e16, -1e16, 1) sum to (0, 1) in ascending
    order, (1, 0) in descending order; with s_j = 1 + 2^-20 and x_j = 1 + 2^-33
    the product 1 + 2^-20 + 2^-33 + 2^-53 rounds to 1 + 2^-20 + 2^-33 (ties
    to even)."""
    A = np.array([[0], [0], [0], [1], [1], [1]], dtype=np.int32)
    x = np.array([1.0, 1e16, -1e16, 1e16, -1e16, 1.0])
    assert orc.measure_scaled(A, 2, np.ones(6), x).tolist() == [0.0, 1.0]
    s1, x1 = 1.0 + 2.0 ** -20, 1.0 + 2.0 ** -33
    y = orc.measure_scaled(np.array([[0]], dtype=np.int32), 1, np.array([s1]), np.array([x1]))
    assert y[0] == 1.0 + 2.0 ** -20 + 2.0 ** -33 and y[0] == s1 * x1


@pytest.mark.parametrize("q,k,seed", [(5, 3, 0), (7, 3, 1), (7, 4, 2)])
def test_scaled_columns_recover_pm1_signals(orc, q, k, seed):
    """Sec. 4.3.3: with every value of x equal to +1 (not dissociated: equal
    values), scaling A's columns by i.i.d. continuous numbers lets
    Parallel-l0 identify the support; decoding y = A (s . x) recovers
    z = s . x exactly in the theorem regime, and z / s = x."""
    rng = np.random.default_rng(300 + 10 * q + seed)
    A = affine_plane(q)
    perm = rng.permutation(q * q).astype(np.int32)
    A = np.sort(perm[A], axis=1).astype(np.int32)
    n, d = A.shape
    m = q * q
    es = eps_star(A, m, k)
    alpha = math.ceil((1 - 2 * es) * d)
    x = np.zeros(n)
    x[np.sort(rng.choice(n, size=k, replace=False))] = 1.0
    s = orc.column_scales(n, 1000 + seed)
    y = orc.measure_scaled(A, m, s, x)
    res = orc.parallel_l0(A, m, y, alpha=alpha, max_iter=50)
    assert res["status"] == orc.CONVERGED
    assert np.array_equal(res["x_hat"], s * x)
    assert np.array_equal(orc.unscale(s, res["x_hat"]), x)


def test_negative_zero_is_zero(orc):
    """||.||_0 counts -0.0 as zero (IEEE -0.0 == 0.0): a measurement of
    signed zeros is already solved by x_hat = 0, and a column whose rows hold
    -0.0 sees no nonzero value to propose."""
    assert orc.l0(np.array([-0.0, 0.0, 1.0, -2.0])) == 2
    A = orc.make_expander(40, 12, 3, 5)
    y = np.full(12, -0.0)
    res = orc.parallel_l0(A, 12, y)
    assert (res["status"], res["iterations"]) == (orc.CONVERGED, 0)
    assert not np.any(res["x_hat"])
    accepted, omega, score, count = orc.score_column(A[0], np.where(np.arange(12) < 6, -0.0, 0.0))
    assert not accepted and (omega, score, count) == (0.0, -3, 0)


def test_repeated_update_accumulates(orc):
    """Alg. 1 and Alg. 2 add omega to x_hat_j (x_hat_j <- x_hat_j + omega),
    so a column accepted twice holds the sum of its updates.  Hand-worked
    instance (count score, alpha = 2, d = 3), columns {0,1,2}, {0,3,4},
    {1,5,6}, y = (1, 1, 5, 2, 2, 2, 2):
      pass 1 accepts all three (omega 1, 2, 2): x_hat = (1, 2, 2),
        r = (-2, -2, 4, 0, 0, 0, 0);
      pass 2 accepts column 0 again with omega = -2: x_hat_0 = 1 - 2 = -1,
        r = (0, 0, 6, 0, 0, 0, 0);
      pass 3 accepts nothing: stalled after 2 iterations.
    Serial-l0 reaches the same state sweep by sweep."""
    A = np.array([[0, 1, 2], [0, 3, 4], [1, 5, 6]], dtype=np.int32)
    y = np.array([1.0, 1.0, 5.0, 2.0, 2.0, 2.0, 2.0])
    for decode in (orc.parallel_l0, orc.serial_l0):
        res = decode(A, 7, y, alpha=2, score_mode=orc.SCORE_COUNT)
        assert (res["status"], res["iterations"]) == (orc.STALLED, 2), decode.__name__
        assert res["x_hat"].tolist() == [-1.0, 2.0, 2.0], decode.__name__
        assert res["r"].tolist() == [0.0, 0.0, 6.0, 0.0, 0.0, 0.0, 0.0], decode.__name__
        assert list(res["r0_hist"]) == [7, 3, 1], decode.__name__


@pytest.mark.parametrize("mode", [0, 1])
def test_shifted_candidate_position_every_iteration(orc, mode):
    """Reading R11 at every iteration of a long shifted decode (100
    iterations, so the position l mod d wraps around many times): with r the
    residual before iteration l, column j is accepted exactly when the value
    w = r at the (l mod d)-th of its ascending rows is nonzero and its score
    reaches alpha, the score taken from its literal definition on the whole
    vector (Eq. 15: ||r||_0 - ||r - w a_j||_0; the count score: the number of
    rows of j holding w); the accepted omega is w."""
    n, m, d = 1500, 150, 3
    p = inputs.make_problem(n, m, d, inputs.round_half_up(0.2 * m), 1)
    A = orc.make_expander(n, m, d, p.a_seed)
    y = orc.measure(A, m, p.x)
    res = orc.parallel_l0(A, m, y, alpha=2, score_mode=mode, shifted=True, trace=True)
    assert res["iterations"] > 2 * d
    dense = np.zeros((n, m))
    dense[np.repeat(np.arange(n), d), A.ravel()] = 1.0
    x_hat = np.zeros(n)
    for it, idx, om in res["trace"]:
        # r before this iteration: y - A x_hat by the residual rule (the count
        # score oscillates to values that are no longer exact on the grid)
        r = orc.residual(A, m, y, x_hat)
        w = r[A[:, it % d]]
        on_rows = r[A] == w[:, None]
        if mode == 0:
            after = r[None, :] - w[:, None] * dense
            score = np.count_nonzero(r) - np.count_nonzero(after, axis=1)
        else:
            score = on_rows.sum(axis=1)
        accept = (w != 0.0) & (score >= 2)
        assert np.array_equal(np.nonzero(accept)[0], idx), it
        assert np.array_equal(om, w[idx]), it
        x_hat[idx] = x_hat[idx] + om
    assert np.array_equal(x_hat, res["x_hat"])


def test_serial_shifted_sweeps_replayed(orc):
    """Reading R11 for Serial-l0 (Alg. 1) over 7 sweeps, so the position
    t mod d wraps around twice.  The state before sweep t is the oracle's
    result with max_iter = t.  The test replays sweep t by the definition:
    columns in order, candidate w = r at the (t mod d)-th ascending row of
    the column, accepted when w != 0 and the literal l0 decrease
    ||r||_0 - ||r - w a_j||_0 reaches alpha, then x_hat_j += w and r = y -
    A x_hat.  The replay must match the oracle with max_iter = t + 1."""
    n, m, d = 1000, 100, 3
    p = inputs.make_problem(n, m, d, inputs.round_half_up(0.2 * m), 2)
    A = orc.make_expander(n, m, d, p.a_seed)
    y = orc.measure(A, m, p.x)
    full = orc.serial_l0(A, m, y, alpha=2, shifted=True, max_iter=40)
    assert full["iterations"] > 2 * d
    x_hat, r = np.zeros(n), y.copy()
    for t in range(full["iterations"]):
        pos = t % d
        for j in range(n):
            w = r[A[j, pos]]
            if w == 0.0:
                continue
            after = r.copy()
            after[A[j]] = after[A[j]] - w
            if np.count_nonzero(r) - np.count_nonzero(after) >= 2:
                x_hat[j] = x_hat[j] + w
                r = orc.residual(A, m, y, x_hat)
        nxt = orc.serial_l0(A, m, y, alpha=2, shifted=True, max_iter=t + 1)
        assert np.array_equal(x_hat, nxt["x_hat"]) and np.array_equal(r, nxt["r"]), t


@pytest.mark.parametrize("serial", [False, True])
def test_shifted_empty_iteration_moves_on(orc, serial):
    """Reading R3 for the shifted variant (Sec. 4.3.1): an iteration whose
    position accepts nothing leaves r unchanged but the next iteration tries
    the next position, so it is counted and the decode goes on.  Columns
    {0,1,2} and {0,3,4} hold x = (1, 2): y = (3, 1, 1, 2, 2).  At position 0
    both candidates are r_0 = 3, which occurs once (score 1 < 2); at
    position 1 the candidates are 1 and 2, which occur on two rows each, and
    both are accepted.  Worked by hand: two iterations, converged, x_hat = x,
    ||r||_0 history (5, 5, 0)."""
    A = np.array([[0, 1, 2], [0, 3, 4]], dtype=np.int32)
    y = np.array([3.0, 1.0, 1.0, 2.0, 2.0])
    decode = orc.serial_l0 if serial else orc.parallel_l0
    res = decode(A, 5, y, alpha=2, shifted=True)
    assert (res["status"], res["iterations"]) == (orc.CONVERGED, 2)
    assert res["x_hat"].tolist() == [1.0, 2.0]
    assert res["r"].tolist() == [0.0] * 5
    assert list(res["r0_hist"]) == [5, 5, 0]
    # the unshifted decode takes the mode (1 on rows 1, 2; 2 on rows 3, 4)
    # and needs no second position
    plain = decode(A, 5, y, alpha=2)
    assert (plain["status"], plain["iterations"]) == (orc.CONVERGED, 1)


@pytest.mark.parametrize("serial", [False, True])
def test_shifted_stalls_after_d_empty_iterations(orc, serial):
    """One column {0,1,2} with r = (1, 2, 3): no value occurs twice, so no
    position is ever accepted.  The shifted decode tries positions 0, 1, 2
    on the same r and stalls when the third empty iteration completes the
    run of d = 3; the first two are counted (history 3, 3, 3).  The
    unshifted decode stalls at once, with no iteration counted."""
    A = np.array([[0, 1, 2]], dtype=np.int32)
    y = np.array([1.0, 2.0, 3.0])
    decode = orc.serial_l0 if serial else orc.parallel_l0
    res = decode(A, 3, y, alpha=2, shifted=True)
    assert (res["status"], res["iterations"]) == (orc.STALLED, 2)
    assert list(res["r0_hist"]) == [3, 3, 3]
    assert res["x_hat"].tolist() == [0.0]
    plain = decode(A, 3, y, alpha=2)
    assert (plain["status"], plain["iterations"]) == (orc.STALLED, 0)
    # with max_iter below the run the cap comes first
    capped = decode(A, 3, y, alpha=2, shifted=True, max_iter=1)
    assert (capped["status"], capped["iterations"]) == (orc.MAX_ITER, 1)

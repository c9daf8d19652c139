"""GPU parity: every output of the CUDA path, called through the C ABI, is
bit-identical to the CPU oracle on the same seeded inputs (tolerance 0:
both sides add in the same order in binary64 and decide equality exactly).
"""
import math

import numpy as np
import pytest

from paper_1508_01256_gb300 import inputs
from gpu_util import assert_same_decode, device_problem, oracle_problem, upload_matrix

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ccs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_01256_gb300 import build, ccs
    build.build()
    return ccs


# ---- generator, transpose, measure -----------------------------------------

EXPANDER_SIZES = [(1, 1, 1), (5, 5, 5), (1000, 97, 1), (1000, 97, 2), (3001, 211, 3),
                  (4096, 410, 7), (777, 16, 16), (20000, 1000, 11), (2 ** 20, 2 ** 17, 7),
                  (2 ** 20, 1049, 9), (65536, 16384, 5), (300000, 2500, 7)]


@pytest.mark.parametrize("n,m,d", EXPANDER_SIZES)
def test_expander_bitwise(ccs, orc, n, m, d):
    seed = 0x5eed0000 + n + 7 * m + d
    csc, ptr, cols = ccs.make_expander(n, m, d, seed)
    A = orc.make_expander(n, m, d, seed)
    assert np.array_equal(csc.cpu().numpy(), A)
    optr, ocols = orc.transpose(A, m)
    assert np.array_equal(ptr.cpu().numpy(), optr)
    assert np.array_equal(cols.cpu().numpy(), ocols)


def test_expander_rejection_branch_bitwise(ccs, orc):
    """Seeds whose column 0 first draws a value Lemire's bounded method must
    reject (a branch random seeds never reach): the device generator takes
    the same next draw as the oracle."""
    import rejection_seeds
    for _, seed in rejection_seeds.rejected_first_draws():
        for n, d in ((1, 1), (3, 2), (40, 5)):
            csc, ptr, cols = ccs.make_expander(n, rejection_seeds.M, d, seed)
            A = orc.make_expander(n, rejection_seeds.M, d, seed)
            assert np.array_equal(csc.cpu().numpy(), A)
            optr, ocols = orc.transpose(A, rejection_seeds.M)
            assert np.array_equal(ptr.cpu().numpy(), optr)
            assert np.array_equal(cols.cpu().numpy(), ocols)


def test_expander_full_extreme_size(ccs, orc):
    """n = 2^24, m = 16777, d = 9: rows of ~9000 columns sorted on chip."""
    n, m, d = 2 ** 24, 16777, 9
    csc, ptr, cols = ccs.make_expander(n, m, d, 99)
    A = orc.make_expander(n, m, d, 99)
    assert np.array_equal(csc.cpu().numpy(), A)
    optr, ocols = orc.transpose(A, m)
    assert np.array_equal(ptr.cpu().numpy(), optr)
    assert np.array_equal(cols.cpu().numpy(), ocols)


@pytest.mark.parametrize("model", ["gauss-grid", "gauss-raw", "pm1"])
@pytest.mark.parametrize("shape", [(4096, 410, 7, 41), (2 ** 20, 2 ** 17, 7, 26214),
                                   (100003, 1001, 9, 300)])
def test_measure_bitwise(ccs, orc, model, shape):
    n, m, d, k = shape
    p = inputs.make_problem(n, m, d, k, 31 + n, model)
    _, _, _, y = device_problem(ccs, p)
    _, y_ref = oracle_problem(orc, p)
    assert np.array_equal(y.cpu().numpy().view(np.int64), y_ref.view(np.int64))


# ---- whole decodes ------------------------------------------------------------

def _decode_both(ccs, orc, p, **kw):
    csc, ptr, cols, y = device_problem(ccs, p)
    g = ccs.decode_parallel_l0(csc, ptr, cols, y, **kw)
    A, y_ref = oracle_problem(orc, p)
    okw = {k: v for k, v in kw.items() if k in ("alpha", "max_iter", "score_mode", "shifted")}
    ref = orc.parallel_l0(A, p.m, y_ref, **okw)
    return g, ref


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("model", ["gauss-grid", "gauss-raw", "pm1"])
def test_decode_small_workload(ccs, orc, seed, model):
    """n=4096, m=410, k=41, d=7."""
    g, ref = _decode_both(ccs, orc, inputs.plain_small(seed=seed, model=model))
    assert_same_decode(g, ref)
    if model == "gauss-grid":
        assert g.status == ccs.CONVERGED


def test_decode_at_scale_grid(ccs, orc):
    """n=2^20, m=2^17, k=26214, d=7: the benchmark workload, compared whole."""
    p = inputs.plain_at_scale(seed=inputs.BASE_SEED)
    g, ref = _decode_both(ccs, orc, p)
    assert_same_decode(g, ref)
    assert g.status == ccs.CONVERGED
    assert np.array_equal(g.x_hat.cpu().numpy(), p.x)


def test_decode_at_scale_raw(ccs, orc):
    p = inputs.plain_at_scale(seed=3, model="gauss-raw")
    g, ref = _decode_both(ccs, orc, p, max_iter=12)
    assert_same_decode(g, ref)


@pytest.mark.parametrize("rho", inputs.EXTREME_RHOS)
def test_decode_extreme_undersampling_scaled(ccs, orc, rho):
    """delta ~ 10^-3, d = 9 at n = 2^20 (the n = 2^24 shape scaled down)."""
    p = inputs.extreme_undersampling(rho, d=9, seed=11, log2n=20)
    g, ref = _decode_both(ccs, orc, p)
    assert_same_decode(g, ref)


def test_decode_extreme_undersampling_full(ccs, orc):
    """n = 2^24, m = 16777, d = 9, rho = 0.05, compared whole."""
    p = inputs.extreme_undersampling(0.05, d=9, seed=5)
    g, ref = _decode_both(ccs, orc, p)
    assert_same_decode(g, ref)
    assert g.status == ccs.CONVERGED


def test_decode_extreme_dense_residual_full(ccs, orc):
    """n = 2^24, m = 16777, d = 9, rho = 0.30 (beyond recovery: r stays
    dense, so most columns pass the zero-count part of the fingerprint bound
    and many reach the exact score), first three iterations compared whole."""
    p = inputs.extreme_undersampling(0.30, d=9, seed=8)
    g, ref = _decode_both(ccs, orc, p, max_iter=3)
    assert_same_decode(g, ref)
    assert g.iterations == 3


@pytest.mark.parametrize("rho,seed", [(0.15, 20151510), (0.20, 20151511), (0.30, 20151513)])
def test_decode_extreme_dense_full_final_state(ccs, orc, rho, seed):
    """n = 2^24, m = 16777, d = 9 past the transition (the bench's seeds):
    the decodes run 64 to 100 iterations, through cascades where hundreds of
    thousands of columns are accepted at once and every row outgrows its
    record, and stall or reach max_iter.  Too long for the oracle to replay
    whole here, so the final state is checked against what the oracle fixes
    at any size: r is the oracle's ordered residual y - A x_hat of the
    returned x_hat, bit for bit; ||r||_0 is the history's last entry; and a
    stalled decode's r is one on which the oracle's score of every column
    accepts none."""
    p = inputs.extreme_undersampling(rho, d=9, seed=seed)
    csc, ptr, cols, y = device_problem(ccs, p)
    g = ccs.decode_parallel_l0(csc, ptr, cols, y)
    assert g.status in (ccs.STALLED, ccs.MAX_ITER) and g.iterations > 3
    A, y_ref = oracle_problem(orc, p)
    assert np.array_equal(y.cpu().numpy().view(np.int64), y_ref.view(np.int64))
    r_ref = orc.residual(A, p.m, y_ref, g.x_hat.cpu().numpy())
    assert np.array_equal(g.r.cpu().numpy().view(np.int64), r_ref.view(np.int64))
    assert g.r0_final == orc.l0(r_ref) == g.r0_hist[-1]
    if g.status == ccs.STALLED:
        acc, _, _ = orc.score_all(A, r_ref)
        assert not acc.any()
    else:
        assert g.iterations == 100


def test_batch_both_fingerprint_widths(ccs, orc):
    """One batch with problems on both sides of the 16-bit fingerprint limit
    (m <= 32768 keeps 16-bit fingerprints, larger m 8-bit ones), d <= 8 and
    d > 8, each equal to the oracle."""
    shapes = [(200000, 60000, 7, 3000), (50000, 5000, 7, 500), (100000, 40000, 9, 2000),
              (30000, 3000, 9, 300), (70000, 32768, 5, 1600), (70000, 32769, 5, 1600)]
    probs = [inputs.make_problem(*sh, seed=900 + i) for i, sh in enumerate(shapes)]
    items = [device_problem(ccs, p) for p in probs]
    outs = ccs.decode_batch(items, history=True)
    for p, g in zip(probs, outs):
        A, y_ref = oracle_problem(orc, p)
        assert_same_decode(g, orc.parallel_l0(A, p.m, y_ref))


def test_decode_extreme_pm1(ccs, orc):
    p = inputs.extreme_undersampling(0.05, d=9, seed=6, model="pm1", log2n=20)
    g, ref = _decode_both(ccs, orc, p)
    assert_same_decode(g, ref)


@pytest.mark.parametrize("d", [2, 3, 5, 8, 11, 13, 16])
@pytest.mark.parametrize("mode", [0, 1])
def test_decode_all_d_and_modes(ccs, orc, d, mode):
    n = 6007  # not a multiple of the block size: ragged tail
    m = max(d, 700)
    p = inputs.make_problem(n, m, d, 70, 900 + d, "gauss-grid")
    for alpha in sorted({2, (d + 1) // 2 + (d % 2 == 0), d}):
        if alpha < 2:
            continue
        g, ref = _decode_both(ccs, orc, p, alpha=alpha, score_mode=mode, max_iter=40)
        assert_same_decode(g, ref)


@pytest.mark.parametrize("d", [5, 7, 9, 12])
def test_parallel_lddsr_matches_oracle(ccs, orc, d):
    """Parallel-LDDSR (Sec. 4.3.2): match-count score, alpha = floor(d/2) + 1,
    on a problem in the regime where it recovers (small rho)."""
    p = inputs.make_problem(40000, 4000, d, 120, 70 + d)
    g, ref = _decode_both(ccs, orc, p, alpha=ccs.lddsr_alpha(d), score_mode=ccs.SCORE_COUNT)
    assert_same_decode(g, ref)


@pytest.mark.parametrize("mode", [0, 1])
def test_alpha_sweep_at_scale(ccs, orc, mode):
    """Every alpha in [2, d] at n = 2^20 (the bench's alpha sweep)."""
    p = inputs.plain_at_scale(seed=23)
    csc, ptr, cols, y = device_problem(ccs, p)
    A, y_ref = oracle_problem(orc, p)
    for alpha in range(2, p.d + 1):
        g = ccs.decode_parallel_l0(csc, ptr, cols, y, alpha=alpha, score_mode=mode, max_iter=30)
        assert_same_decode(g, orc.parallel_l0(A, p.m, y_ref, alpha=alpha, score_mode=mode,
                                              max_iter=30))


def test_first_iteration_is_the_score_step(ccs, orc):
    """max_iter = 1: x_hat equals omega_j on the accepted columns of one score
    pass over r = y (Eq. (15) with the tie rule), zero elsewhere."""
    p = inputs.plain_small(seed=4)
    g, ref = _decode_both(ccs, orc, p, max_iter=1)
    assert_same_decode(g, ref)
    A, y_ref = oracle_problem(orc, p)
    acc, om, _ = orc.score_all(A, y_ref)
    expect = np.where(acc, om, 0.0)
    assert np.array_equal(g.x_hat.cpu().numpy(), expect)


def test_edge_k0(ccs, orc):
    p = inputs.make_problem(3000, 300, 7, 0, 1)
    g, ref = _decode_both(ccs, orc, p)
    assert_same_decode(g, ref)
    assert g.status == ccs.CONVERGED and g.iterations == 0


def test_edge_max_iter_zero(ccs, orc):
    g, ref = _decode_both(ccs, orc, inputs.plain_small(seed=1), max_iter=0)
    assert_same_decode(g, ref)
    assert g.status == ccs.MAX_ITER


def test_edge_tiny_shapes(ccs, orc):
    for (n, m, d, k) in [(1, 2, 2, 1), (2, 2, 2, 1), (7, 3, 3, 2), (33, 5, 4, 3), (257, 16, 16, 5)]:
        p = inputs.make_problem(n, m, d, k, n * 31 + m)
        g, ref = _decode_both(ccs, orc, p, alpha=2)
        assert_same_decode(g, ref)


def test_edge_stalled(ccs, orc):
    import torch
    A = np.array([[0, 1, 2], [2, 3, 4]], dtype=np.int32)
    csc, ptr, cols = upload_matrix(orc, A, 5)
    y = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    g = ccs.decode_parallel_l0(csc, ptr, cols, torch.from_numpy(y).cuda(), alpha=2)
    ref = orc.parallel_l0(A, 5, y)
    assert_same_decode(g, ref)
    assert g.status == ccs.STALLED


def test_edge_count_mode_oscillation(ccs, orc):
    import torch
    A = np.array([[0, 1, 2], [0, 1, 3], [2, 3, 4]], dtype=np.int32)
    csc, ptr, cols = upload_matrix(orc, A, 5)
    y = np.array([0.5, 0.5, 0.5, 0.0, 0.0])
    for mode in (0, 1):
        g = ccs.decode_parallel_l0(csc, ptr, cols, torch.from_numpy(y).cuda(), alpha=2,
                                   score_mode=mode, max_iter=9)
        ref = orc.parallel_l0(A, 5, y, alpha=2, score_mode=mode, max_iter=9)
        assert_same_decode(g, ref)


def test_edge_slot_overflow_rows(ccs, orc):
    """Rows with more than 15 nonzero contributors take the whole-row path."""
    n, m, d = 4000, 60, 7   # k d / m ~ 47 contributors per row
    p = inputs.make_problem(n, m, d, 400, 77)
    g, ref = _decode_both(ccs, orc, p, max_iter=20)
    assert_same_decode(g, ref)


@pytest.mark.parametrize("flags", [2, 4])
def test_overflow_rows_under_ordered_residual(ccs, orc, flags):
    """Rows of up to ~50 nonzero contributors under the ordered residual
    (bit 1: from the first iteration; bit 2: from iteration 2), so their
    sums walk the whole CSR row: bit-identical to the oracle."""
    n, m, d = 4000, 60, 7
    p = inputs.make_problem(n, m, d, 400, 77)
    g, ref = _decode_both(ccs, orc, p, max_iter=20, debug_flags=flags)
    assert_same_decode(g, ref)


def _affine_plane(q):
    lines = [sorted(a * q + (s * a + c) % q for a in range(q)) for s in range(q) for c in range(q)]
    lines += [sorted(c * q + b for b in range(q)) for c in range(q)]
    return np.array(lines, dtype=np.int32)


@pytest.mark.parametrize("seed", range(3))
def test_theorem_regime_on_gpu(ccs, orc, seed):
    """AG(2,7) incidence (eps < 1/4 for k <= 4, alpha = 4): exact recovery,
    bit-identical to the oracle."""
    import torch
    rng = np.random.default_rng(seed)
    A = _affine_plane(7)
    perm = rng.permutation(49).astype(np.int32)
    A = np.sort(perm[A], axis=1).astype(np.int32)
    x = np.zeros(A.shape[0])
    supp = rng.choice(A.shape[0], size=4, replace=False)
    x[supp] = inputs.values(4, seed, "gauss-grid")
    y = orc.measure(A, 49, x)
    csc, ptr, cols = upload_matrix(orc, A, 49)
    g = ccs.decode_parallel_l0(csc, ptr, cols, torch.from_numpy(y).cuda(), alpha=4)
    ref = orc.parallel_l0(A, 49, y, alpha=4)
    assert_same_decode(g, ref)
    assert np.array_equal(g.x_hat.cpu().numpy(), x)


def test_repeated_update_accumulates_on_gpu(ccs, orc):
    """The hand-worked instance of the oracle pin (count score, alpha = 2):
    column 0 is accepted in two iterations and x_hat_0 = 1 + (-2) = -1,
    bit-identical to the oracle."""
    import torch
    A = np.array([[0, 1, 2], [0, 3, 4], [1, 5, 6]], dtype=np.int32)
    y = np.array([1.0, 1.0, 5.0, 2.0, 2.0, 2.0, 2.0])
    csc, ptr, cols = upload_matrix(orc, A, 7)
    g = ccs.decode_parallel_l0(csc, ptr, cols, torch.from_numpy(y).cuda(), alpha=2,
                               score_mode=ccs.SCORE_COUNT)
    ref = orc.parallel_l0(A, 7, y, alpha=2, score_mode=orc.SCORE_COUNT)
    assert_same_decode(g, ref)
    assert g.x_hat.cpu().numpy().tolist() == [-1.0, 2.0, 2.0]


@pytest.mark.parametrize("case", ["moves_on", "stalls"])
def test_shifted_empty_iterations_on_gpu(ccs, orc, case):
    """The hand-worked instances of the oracle pins on the shifted stall rule
    (Sec. 4.3.1): an iteration that accepts nothing moves to the next
    position and is counted; d of them in a row stall the decode.  Alone and
    in a batch (where the run length persists across the launches that
    merge the groups' tails), bit-identical to the oracle."""
    import torch
    if case == "moves_on":
        A = np.array([[0, 1, 2], [0, 3, 4]], dtype=np.int32)
        y = np.array([3.0, 1.0, 1.0, 2.0, 2.0])
        want = (orc.CONVERGED, 2, [5, 5, 0])
    else:
        A = np.array([[0, 1, 2]], dtype=np.int32)
        y = np.array([1.0, 2.0, 3.0])
        want = (orc.STALLED, 2, [3, 3, 3])
    m = y.size
    csc, ptr, cols = upload_matrix(orc, A, m)
    yd = torch.from_numpy(y).cuda()
    ref = orc.parallel_l0(A, m, y, alpha=2, shifted=True)
    assert (ref["status"], ref["iterations"], list(ref["r0_hist"])) == want
    g = ccs.decode_parallel_l0(csc, ptr, cols, yd, alpha=2, shifted=True)
    assert_same_decode(g, ref)
    big = inputs.make_problem(20000, 2000, 3, 400, 77)
    items = [(csc, ptr, cols, yd), device_problem(ccs, big)]
    outs = ccs.decode_batch(items, history=True, shifted=True)
    assert_same_decode(outs[0], ref)
    A2, y2 = oracle_problem(orc, big)
    assert_same_decode(outs[1], orc.parallel_l0(A2, big.m, y2, shifted=True))


@pytest.mark.parametrize("case", ["y_zero", "max_iter_zero"])
def test_decode_stopping_at_once_zeroes_dirty_x_hat(ccs, orc, case):
    """A lone problem's x_hat <- 0 is stored by its first score phase; a
    decode that stops before one (y = 0, or max_iter = 0) zeroes x_hat after
    the init barrier.  Outputs filled with NaN beforehand come back equal to
    the oracle's, twice on the same buffers."""
    import torch
    p = inputs.make_problem(4096, 410, 7, 0 if case == "y_zero" else 41, 5)
    kw = {"max_iter": 0} if case == "max_iter_zero" else {}
    csc, ptr, cols, y = device_problem(ccs, p)
    A, y_ref = oracle_problem(orc, p)
    ref = orc.parallel_l0(A, p.m, y_ref, **kw)
    x_hat = torch.full((p.n,), float("nan"), dtype=torch.float64, device="cuda")
    r = torch.full((p.m,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        g = ccs.decode_parallel_l0(csc, ptr, cols, y, out=(x_hat, r, None), **kw)
        assert_same_decode(g, ref, check_hist=False)
        assert g.iterations == 0
        x_hat.fill_(float("nan"))


def test_workspace_reuse_and_dirty_outputs(ccs, orc):
    """A reused workspace and garbage in the output buffers change nothing."""
    import torch
    p = inputs.plain_small(seed=9)
    csc, ptr, cols, y = device_problem(ccs, p)
    ws = ccs.workspace(ccs.ccs_workspace_size(ccs.OP_DECODE, p.n, p.m, p.d))
    ws.fill_(0xAB)
    x_hat = torch.full((p.n,), float("nan"), dtype=torch.float64, device="cuda")
    r = torch.full((p.m,), 3.0, dtype=torch.float64, device="cuda")
    hist = torch.full((101,), -7, dtype=torch.int64, device="cuda")
    A, y_ref = oracle_problem(orc, p)
    ref = orc.parallel_l0(A, p.m, y_ref)
    for _ in range(2):
        g = ccs.decode_parallel_l0(csc, ptr, cols, y, ws=ws, out=(x_hat, r, hist))
        assert_same_decode(g, ref)


def test_batch_equals_single(ccs, orc):
    probs = [inputs.make_problem(*shape, seed=300 + i) for i, shape in enumerate(
        [(4096, 410, 7, 41), (1000, 100, 5, 20), (20000, 2000, 9, 400), (5000, 50, 11, 5)])]
    items = [device_problem(ccs, p) for p in probs]
    outs = ccs.decode_batch(items, history=True)
    for p, (csc, ptr, cols, y), g in zip(probs, items, outs):
        single = ccs.decode_parallel_l0(csc, ptr, cols, y)
        assert g.status == single.status and g.iterations == single.iterations
        assert g.r0_hist == single.r0_hist
        assert np.array_equal(g.x_hat.cpu().numpy(), single.x_hat.cpu().numpy())
        A, y_ref = oracle_problem(orc, p)
        assert_same_decode(g, orc.parallel_l0(A, p.m, y_ref))


def test_iterations_within_log_k(ccs):
    """Sec. 5.4: iterations grow like log k (soft: <= ln k + 2 on exact
    recovery at n = 2^20, delta = 0.1, d = 7, rho in [0.05, 0.1])."""
    for rho in (0.05, 0.075, 0.1):
        m = round(0.1 * 2 ** 20)
        k = inputs.round_half_up(rho * m)
        p = inputs.make_problem(2 ** 20, m, 7, k, 4242)
        csc, ptr, cols, y = device_problem(ccs, p)
        g = ccs.decode_parallel_l0(csc, ptr, cols, y)
        assert g.status == ccs.CONVERGED
        assert g.iterations <= math.log(k) + 2


# ---- engines -------------------------------------------------------------------

@pytest.mark.parametrize("engine", [1, 3])
@pytest.mark.parametrize("shape", [(4096, 410, 7, 41), (2 ** 20, 2 ** 17, 7, 26214),
                                   (300000, 300, 9, 30), (5000, 250000, 5, 2000),
                                   (60001, 6000, 16, 900)])
def test_engines_match_oracle(ccs, orc, engine, shape):
    """Host-driven loop and persistent engine, each bit-identical to the
    oracle; the last two shapes take the no-fingerprint path (m too large
    for shared memory) and the 512-thread d=16 engine."""
    n, m, d, k = shape
    p = inputs.make_problem(n, m, d, k, 4000 + n % 97)
    g, ref = _decode_both(ccs, orc, p, engine=engine)
    assert_same_decode(g, ref)


RESIDUAL_CASES = [("small", lambda: inputs.plain_small(seed=3)),
                  ("small-raw", lambda: inputs.plain_small(seed=3, model="gauss-raw")),
                  ("small-pm1", lambda: inputs.plain_small(seed=3, model="pm1")),
                  ("extreme-scaled", lambda: inputs.extreme_undersampling(0.25, d=9, seed=13,
                                                                          log2n=20)),
                  ("mid", lambda: inputs.make_problem(200000, 20000, 7, 4000, 17))]


@pytest.mark.parametrize("flags", [0, 2, 4])
@pytest.mark.parametrize("case", [c[0] for c in RESIDUAL_CASES])
def test_residual_modes_match_oracle(ccs, orc, case, flags):
    """The persistent engine keeps r by exact atomic updates while its
    certificate holds, else by ordered row sums; debug bit 1 forces the
    ordered form from the start, bit 2 a switch at iteration 2 (its records
    rebuilt on the way).  Every form equals the oracle bit for bit, and the
    result reports the form the decode ended in."""
    p = dict(RESIDUAL_CASES)[case]()
    g, ref = _decode_both(ccs, orc, p, engine=ccs.ENGINE_PERSISTENT, debug_flags=flags,
                          max_iter=40)
    assert_same_decode(g, ref)
    if flags == 2 or (flags == 4 and g.iterations > 2):
        assert g.residual_form == ccs.RESIDUAL_ORDERED
    elif flags == 0 and p.model == "gauss-grid" and g.status == ccs.CONVERGED:
        assert g.residual_form == ccs.RESIDUAL_EXACT


def test_residual_mode_switch_in_batch(ccs, orc):
    """A batch where the certificate fails at iteration 2 for every problem:
    each result still equals the oracle."""
    probs = inputs.batch_problems(12, seed=31, log2n_hi=15.0)
    items = [device_problem(ccs, p) for p in probs]
    outs = ccs.decode_batch(items, history=True, debug_flags=4)
    for p, g in zip(probs, outs):
        A, y_ref = oracle_problem(orc, p)
        assert_same_decode(g, orc.parallel_l0(A, p.m, y_ref))


def test_watchdog_times_out_and_context_survives(ccs, orc):
    """Test hook: CTA 0 never arrives at the first score barrier, so every
    CTA's bounded wait runs out (200 ms); the call reports CCS_ETIMEOUT and
    the next decode on the same context is correct."""
    p = inputs.plain_small(seed=12)
    csc, ptr, cols, y = device_problem(ccs, p)
    with pytest.raises(ccs.CcsError) as ei:
        ccs.decode_parallel_l0(csc, ptr, cols, y, engine=ccs.ENGINE_PERSISTENT,
                               watchdog_ms=200, debug_flags=1)
    assert ei.value.code == ccs.CCS_ETIMEOUT
    g = ccs.decode_parallel_l0(csc, ptr, cols, y, engine=ccs.ENGINE_PERSISTENT)
    A, y_ref = oracle_problem(orc, p)
    assert_same_decode(g, orc.parallel_l0(A, p.m, y_ref))


@pytest.mark.parametrize("engine", [1, 3])
def test_mixed_batch_matches_oracle(ccs, orc, engine):
    """A mixed batch (n log-uniform in [2^12, 2^16], delta, rho, d drawn as in
    the batched workload) in one call equals the oracle problem by problem."""
    probs = inputs.batch_problems(40, seed=77, log2n_hi=16.0)
    items = [device_problem(ccs, p) for p in probs]
    outs = ccs.decode_batch(items, history=True, engine=engine)
    for p, g in zip(probs, outs):
        A, y_ref = oracle_problem(orc, p)
        assert_same_decode(g, orc.parallel_l0(A, p.m, y_ref))


def test_batch_order_does_not_matter(ccs):
    probs = inputs.batch_problems(12, seed=5, log2n_hi=15.0)
    items = [device_problem(ccs, p) for p in probs]
    fwd = ccs.decode_batch(items)
    rev = ccs.decode_batch(items[::-1])[::-1]
    for a, b in zip(fwd, rev):
        assert a.status == b.status and a.iterations == b.iterations
        assert np.array_equal(a.x_hat.cpu().numpy(), b.x_hat.cpu().numpy())
        assert np.array_equal(a.r.cpu().numpy(), b.r.cpu().numpy())


def test_async_decode_matches_blocking(ccs, orc):
    """ccs_decode_parallel_l0_async: results land in device memory, several
    decodes queued back to back on one stream without a host wait."""
    import torch
    probs = [inputs.plain_small(seed=s) for s in range(3)] + \
        [inputs.make_problem(50000, 5000, 9, 600, 71)]
    items = [device_problem(ccs, p) for p in probs]
    res_dev = ccs.result_buffer(len(probs))
    outs = []
    for i, (p, (csc, ptr, cols, y)) in enumerate(zip(probs, items)):
        x_hat = torch.empty(p.n, dtype=torch.float64, device="cuda")
        r = torch.empty(p.m, dtype=torch.float64, device="cuda")
        ws = ccs.workspace(ccs.ccs_workspace_size(ccs.OP_DECODE, p.n, p.m, p.d))
        ccs.ccs_decode_parallel_l0_async(p.n, p.m, p.d, csc, ptr, cols, y, x_hat, r, None,
                                         ccs.params(), res_dev[i * ccs.RESULT_BYTES:], ws)
        outs.append((x_hat, r, ws))
    torch.cuda.synchronize()
    res = ccs.results_from_device(res_dev, len(probs))
    for p, (x_hat, r, _), rr in zip(probs, outs, res):
        A, y_ref = oracle_problem(orc, p)
        ref = orc.parallel_l0(A, p.m, y_ref)
        assert rr.error == 0 and rr.status == ref["status"]
        assert rr.iterations == ref["iterations"] and rr.r0_final == ref["r0_final"]
        assert np.array_equal(x_hat.cpu().numpy(), ref["x_hat"])
        assert np.array_equal(r.cpu().numpy(), ref["r"])


def test_async_batch_matches_oracle(ccs, orc):
    import torch
    probs = inputs.batch_problems(16, seed=91, log2n_hi=15.0)
    # both d classes: two launches, results written to interleaved slots
    assert {p.d > 8 for p in probs} == {True, False}
    items = [device_problem(ccs, p) for p in probs]
    pbs, outs = [], []
    for (csc, ptr, cols, y), p in zip(items, probs):
        x_hat = torch.empty(p.n, dtype=torch.float64, device="cuda")
        r = torch.empty(p.m, dtype=torch.float64, device="cuda")
        outs.append((x_hat, r))
        pbs.append(ccs.problem(csc, ptr, cols, y, x_hat, r))
    ws = ccs.workspace(ccs.ccs_batch_workspace_size(pbs))
    res_dev = ccs.result_buffer(len(pbs))
    ccs.ccs_decode_batch_async(pbs, ccs.params(), res_dev, ws)
    torch.cuda.synchronize()
    for p, (x_hat, r), rr in zip(probs, outs, ccs.results_from_device(res_dev, len(pbs))):
        A, y_ref = oracle_problem(orc, p)
        ref = orc.parallel_l0(A, p.m, y_ref)
        assert rr.error == 0 and rr.status == ref["status"] and rr.iterations == ref["iterations"]
        assert np.array_equal(x_hat.cpu().numpy(), ref["x_hat"])


def test_async_watchdog_reports_on_device(ccs):
    import torch
    p = inputs.plain_small(seed=3)
    csc, ptr, cols, y = device_problem(ccs, p)
    x_hat = torch.empty(p.n, dtype=torch.float64, device="cuda")
    r = torch.empty(p.m, dtype=torch.float64, device="cuda")
    ws = ccs.workspace(ccs.ccs_workspace_size(ccs.OP_DECODE, p.n, p.m, p.d))
    res_dev = ccs.result_buffer(1)
    ccs.ccs_decode_parallel_l0_async(p.n, p.m, p.d, csc, ptr, cols, y, x_hat, r, None,
                                     ccs.params(watchdog_ms=100, debug_flags=1), res_dev, ws)
    torch.cuda.synchronize()
    assert ccs.results_from_device(res_dev, 1)[0].error == ccs.CCS_ETIMEOUT


def test_binding_checks_arrays_before_the_library(ccs):
    """Wrong dtypes, sizes, non-contiguous views and a history shorter than
    max_iter + 1 are refused in Python, before any pointer reaches the
    library."""
    import torch
    p = inputs.plain_small()
    csc, ptr, cols, y = device_problem(ccs, p)
    x_hat = torch.empty(p.n, dtype=torch.float64, device="cuda")
    r = torch.empty(p.m, dtype=torch.float64, device="cuda")
    short = torch.empty(50, dtype=torch.int64, device="cuda")
    with pytest.raises(ValueError, match="r0_hist"):
        ccs.decode_parallel_l0(csc, ptr, cols, y, out=(x_hat, r, short))  # max_iter 100
    with pytest.raises(ValueError, match="x_hat"):
        ccs.problem(csc, ptr, cols, y, x_hat.float(), r)
    with pytest.raises(ValueError, match="r"):
        ccs.problem(csc, ptr, cols, y, x_hat, r[:-1])
    with pytest.raises(ValueError, match="y"):
        ccs.problem(csc, ptr, cols, torch.stack([y, y], 1)[:, 0], x_hat, r)  # strided view
    with pytest.raises(TypeError, match="ws"):
        ccs.decode_parallel_l0(csc, ptr, cols, y, ws=torch.empty(1 << 20, dtype=torch.uint8))
    ccs.problem(csc, ptr, cols, y, x_hat, r, torch.empty(101, dtype=torch.int64, device="cuda"),
                max_iter=100)  # long enough


def test_batch_graph_replays(ccs, orc):
    """A batched decode captured in a CUDA graph: replays equal
    ccs_decode_batch, and writing new measurements y in place then replaying
    decodes the new signals (each against the oracle)."""
    import torch
    probs = inputs.batch_problems(10, seed=123, log2n_hi=15.0)
    assert {p.d > 8 for p in probs} == {True, False}  # two groups and the merged tail
    items = [device_problem(ccs, p) for p in probs]
    outs, pbs = [], []
    for (csc, ptr, cols, y), p in zip(items, probs):
        x_hat = torch.empty(p.n, dtype=torch.float64, device="cuda")
        r = torch.empty(p.m, dtype=torch.float64, device="cuda")
        outs.append((x_hat, r))
        pbs.append(ccs.problem(csc, ptr, cols, y, x_hat, r))
    g = ccs.BatchGraph(pbs, ccs.params())
    ref = ccs.decode_batch(items)
    for _ in range(2):
        g.launch()
        torch.cuda.synchronize()
        for (x_hat, r), rr, res in zip(outs, ref, g.read_results()):
            assert res.status == rr.status and res.iterations == rr.iterations
            assert torch.equal(x_hat, rr.x_hat) and torch.equal(r, rr.r)
    # new signals on the same matrices, measured into the same y buffers
    new = [inputs.make_problem(p.n, p.m, p.d, p.k, p.seed + 999) for p in probs]
    for (csc, ptr, cols, y), p, q in zip(items, probs, new):
        y.copy_(ccs.measure(ptr, cols, torch.from_numpy(q.x).cuda(), p.m, p.d))
    g.launch()
    torch.cuda.synchronize()
    for (csc, ptr, cols, y), p, q, (x_hat, r), res in zip(items, probs, new, outs,
                                                          g.read_results()):
        A = orc.make_expander(p.n, p.m, p.d, p.a_seed)
        oref = orc.parallel_l0(A, p.m, orc.measure(A, p.m, q.x))
        assert res.status == oref["status"] and res.iterations == oref["iterations"]
        assert np.array_equal(x_hat.cpu().numpy(), oref["x_hat"])
    g.close()


def test_autotune_records_a_shape_and_keeps_results(ccs, orc):
    """ccs_autotune times every launch shape of each launch group and records
    the fastest; decodes that follow (schedule 0) use it and still equal the
    oracle bit for bit."""
    import torch
    probs = inputs.batch_problems(12, seed=57, log2n_hi=15.0)
    assert {p.d > 8 for p in probs} == {True, False}
    items = [device_problem(ccs, p) for p in probs]
    pbs = []
    for (csc, ptr, cols, y), p in zip(items, probs):
        x_hat = torch.empty(p.n, dtype=torch.float64, device="cuda")
        r = torch.empty(p.m, dtype=torch.float64, device="cuda")
        pbs.append(ccs.problem(csc, ptr, cols, y, x_hat, r))
    ws = ccs.workspace(ccs.ccs_batch_workspace_size(pbs))
    try:
        tuned = ccs.ccs_autotune(pbs, ccs.params(), ws)
        torch.cuda.synchronize()
        groups = [t for t in tuned if t]
        # thread shape 1..3, stage cap 0 or 2..3, queue cap 0..1
        assert len(groups) >= 2 and all(
            (t & 3) in (1, 2, 3) and (t >> 2) & 7 in (0, 2, 3) and (t >> 5) in (0, 1)
            for t in groups)
        outs = ccs.decode_batch(items, history=True)
        for p, g in zip(probs, outs):
            A, y_ref = oracle_problem(orc, p)
            assert_same_decode(g, orc.parallel_l0(A, p.m, y_ref))
    finally:
        ccs.ccs_autotune_reset()


@pytest.mark.parametrize("schedule", [1 | (2 << 2), 3 | (3 << 2) | (1 << 5), 2 | (6 << 2),
                                      2 | (2 << 5), 1 | (1 << 5)])
def test_explicit_launch_shapes_keep_results(ccs, orc, schedule):
    """Stage and queue caps change the launch, never the decode: one problem
    per d class, bit for bit against the oracle under each shape (d > 8 takes
    the 512-thread instance whatever the thread shape asks)."""
    for p in (inputs.make_problem(20000, 2000, 7, 400, 61),
              inputs.make_problem(20000, 2000, 11, 300, 62)):
        csc, ptr, cols, y = device_problem(ccs, p)
        A, y_ref = oracle_problem(orc, p)
        g = ccs.decode_parallel_l0(csc, ptr, cols, y, schedule=schedule)
        assert_same_decode(g, orc.parallel_l0(A, p.m, y_ref))


def test_autotune_table_round_trips_through_a_file(ccs, tmp_path):
    """ccs_autotune_save / ccs_autotune_load: the recorded shapes come back
    for this GPU model after a reset; lines for other GPUs or malformed ones
    are ignored."""
    import torch
    probs = inputs.batch_problems(6, seed=58, log2n_hi=14.0, ds=(7,))
    pbs, keep = [], []
    for p in probs:
        csc, ptr, cols, y = device_problem(ccs, p)
        x_hat = torch.empty(p.n, dtype=torch.float64, device="cuda")
        r = torch.empty(p.m, dtype=torch.float64, device="cuda")
        keep.append((csc, ptr, cols, y, x_hat, r))
        pbs.append(ccs.problem(csc, ptr, cols, y, x_hat, r))
    ws = ccs.workspace(ccs.ccs_batch_workspace_size(pbs))
    path = str(tmp_path / "shapes.txt")
    try:
        tuned = [t for t in ccs.ccs_autotune(pbs, ccs.params(), ws) if t]
        assert tuned
        want = ccs.ccs_autotune_get(7, True)
        assert want == tuned[0]
        ccs.ccs_autotune_save(path)
        with open(path, "a") as f:
            f.write("Some_Other_GPU/sm1/cc1.0 7 1 9\nnot a line\n")
        ccs.ccs_autotune_reset()
        assert ccs.ccs_autotune_get(7, True) == 0
        ccs.ccs_autotune_load(path)
        assert ccs.ccs_autotune_get(7, True) == want
    finally:
        ccs.ccs_autotune_reset()


SHIFTED_CASES = [(4096, 410, 7, 41, 0), (6007, 700, 5, 70, 1), (20000, 2000, 9, 300, 0),
                 (60001, 6000, 16, 500, 1), (2 ** 20, 2 ** 17, 7, 13107, 0)]


@pytest.mark.parametrize("shape", SHIFTED_CASES)
def test_shifted_matches_oracle(ccs, orc, shape):
    """Shifted Parallel-l0 (Sec. 4.3.1): at iteration l the candidate of
    each column is r at its (l mod d)-th row; bit-identical to the oracle."""
    n, m, d, k, mode = shape
    p = inputs.make_problem(n, m, d, k, 500 + d)
    for alpha in sorted({2, d // 2 + 1, d}):
        g, ref = _decode_both(ccs, orc, p, alpha=alpha, score_mode=mode, max_iter=60,
                              shifted=True)
        assert_same_decode(g, ref)


def test_shifted_batch_and_residual_modes(ccs, orc):
    """Shifted variant in a mixed batch, with the exact residual and with a
    forced switch to the ordered residual."""
    probs = inputs.batch_problems(10, seed=19, log2n_hi=15.0)
    items = [device_problem(ccs, p) for p in probs]
    for flags in (0, 4):
        outs = ccs.decode_batch(items, history=True, shifted=True, debug_flags=flags)
        for p, g in zip(probs, outs):
            A, y_ref = oracle_problem(orc, p)
            assert_same_decode(g, orc.parallel_l0(A, p.m, y_ref, shifted=True))


def test_shifted_rejected_on_host_loop(ccs):
    p = inputs.plain_small(seed=2)
    csc, ptr, cols, y = device_problem(ccs, p)
    with pytest.raises(ccs.CcsError) as ei:
        ccs.decode_parallel_l0(csc, ptr, cols, y, engine=ccs.ENGINE_HOST_LOOP, shifted=True)
    assert ei.value.code == ccs.CCS_EINVAL


@pytest.mark.parametrize("n,seed", [(1, 3), (1000, 7), (2 ** 20 + 13, 99)])
def test_column_scales_bitwise(ccs, orc, n, seed):
    s = ccs.column_scales(n, seed)
    assert np.array_equal(s.cpu().numpy(), orc.column_scales(n, seed))


@pytest.mark.parametrize("shape", [(4096, 410, 7, 41), (2 ** 20, 1049, 9, 52),
                                   (100000, 10000, 16, 800)])
def test_scaled_pipeline_matches_oracle(ccs, orc, shape):
    """Sec. 4.3.3 with +/-1 signals (not dissociated): scales, y = A diag(s) x,
    Parallel-l0 decode of z = s . x, and x = z / s, each bit-identical to the
    oracle; the decode recovers x exactly."""
    import torch
    n, m, d, k = shape
    p = inputs.make_problem(n, m, d, k, 77 + d, "pm1")
    A = orc.make_expander(n, m, d, p.a_seed)
    csc, ptr, cols = upload_matrix(orc, A, m)
    s = ccs.column_scales(n, 4242)
    s_ref = orc.column_scales(n, 4242)
    assert np.array_equal(s.cpu().numpy(), s_ref)
    y = ccs.measure_scaled(ptr, cols, s, torch.from_numpy(p.x).cuda(), m, d)
    y_ref = orc.measure_scaled(A, m, s_ref, p.x)
    assert np.array_equal(y.cpu().numpy(), y_ref)
    g = ccs.decode_parallel_l0(csc, ptr, cols, y)
    ref = orc.parallel_l0(A, m, y_ref)
    assert_same_decode(g, ref)
    x = ccs.unscale(s, g.x_hat)
    assert np.array_equal(x.cpu().numpy(), orc.unscale(s_ref, ref["x_hat"]))
    if n >= 4096:
        assert g.status == ccs.CONVERGED and np.array_equal(x.cpu().numpy(), p.x)


# ---- row-driven score phase ----------------------------------------------------
#
# Once ||r||_0 is small the engine finds the columns that can still be
# accepted from the CSR rows of the nonzero r_i instead of streaming every
# column.  Nothing may change: every decode below is compared bit for bit
# with the oracle, with the phase taken as the engine chooses, forced
# whenever its row list fits (bit 4), with its candidates scored one by one
# (bit 3), and never (bit 5).

ROW_ALWAYS, ROW_INLINE, ROW_NEVER = 16, 8, 32


@pytest.mark.parametrize("case", ["extreme_2e22", "at_scale", "count", "shifted", "alpha3",
                                  "ordered", "switch"])
def test_row_driven_phase_matches_oracle(ccs, orc, case):
    if case == "at_scale":
        p = inputs.plain_at_scale(seed=41)
    else:
        p = inputs.extreme_undersampling(0.08, d=7, seed=42, log2n=22)
    kw = dict(count=dict(score_mode=ccs.SCORE_COUNT, alpha=3),
              shifted=dict(shifted=True), alpha3=dict(alpha=3),
              ordered=dict(debug_flags=2), switch=dict(debug_flags=4)).get(case, {})
    okw = {k: v for k, v in kw.items() if k != "debug_flags"}
    if "score_mode" in okw:
        okw["score_mode"] = orc.SCORE_COUNT
    csc, ptr, cols, y = device_problem(ccs, p)
    A, y_ref = oracle_problem(orc, p)
    ref = orc.parallel_l0(A, p.m, y_ref, **okw)
    seen_rows = False
    for extra in (0, ROW_ALWAYS, ROW_ALWAYS | ROW_INLINE, ROW_NEVER):
        flags = kw.get("debug_flags", 0) | extra
        g = ccs.decode_parallel_l0(csc, ptr, cols, y, **dict(kw, debug_flags=flags))
        assert_same_decode(g, ref)
        if extra & ROW_NEVER:
            assert g.row_driven == 0 and g.row_entries == 0
        seen_rows |= g.row_driven > 0
    assert seen_rows, "no decode took the row-driven phase"


def test_row_driven_entries_count(ccs, orc):
    """row_entries is the number of CSR entries of the nonzero rows summed
    over the row-driven iterations: recomputed here from the oracle's
    residuals, iteration by iteration, with the phase forced."""
    p = inputs.extreme_undersampling(0.05, d=7, seed=43, log2n=22)
    csc, ptr, cols, y = device_problem(ccs, p)
    A, y_ref = oracle_problem(orc, p)
    g = ccs.decode_parallel_l0(csc, ptr, cols, y, debug_flags=ROW_ALWAYS)
    ref = orc.parallel_l0(A, p.m, y_ref, trace=True)
    assert_same_decode(g, ref)
    # a converged decode ran a score phase for exactly its traced iterations
    assert ref["status"] == orc.CONVERGED and len(ref["trace"]) == ref["iterations"]
    deg = np.diff(orc.transpose(A, p.m)[0])
    x_hat = np.zeros(p.n)
    want, iters = 0, 0
    for it, idx, om in ref["trace"]:
        r = orc.residual(A, p.m, y_ref, x_hat)
        if it >= 1:  # the first iteration always streams the columns
            want += int(deg[r != 0.0].sum())
            iters += 1
        x_hat[idx] = x_hat[idx] + om
    assert g.row_driven == iters and g.row_entries == want


@pytest.mark.parametrize("m", [4195, 4197, 40001, 40003])
def test_row_driven_after_dirty_workspace(ccs, orc, m):
    """The per-column counters live in the workspace: garbage there, and a
    second decode on the same workspace, change nothing.  m is odd, so the
    last word of the fingerprints (16-bit up to m = 32768, 8-bit above)
    holds padding that the nonzero-row listing must skip."""
    import torch
    p = inputs.make_problem(2 ** 22, m, 7, inputs.round_half_up(0.05 * m), 44)
    csc, ptr, cols, y = device_problem(ccs, p)
    ws = ccs.workspace(ccs.ccs_workspace_size(ccs.OP_DECODE, p.n, p.m, p.d))
    ws.fill_(0x5A)
    A, y_ref = oracle_problem(orc, p)
    ref = orc.parallel_l0(A, p.m, y_ref)
    for _ in range(2):
        g = ccs.decode_parallel_l0(csc, ptr, cols, y, ws=ws, debug_flags=ROW_ALWAYS)
        assert_same_decode(g, ref)
        assert g.row_driven >= 1


@pytest.mark.parametrize("case", ["small", "extreme_2e22", "count", "shifted", "ordered"])
def test_stream_candidates_scored_inline_match_oracle(ccs, orc, case):
    """Debug bit 6 scores every candidate of the column stream where it is
    found instead of queueing it (the path a full queue takes): the decode
    is the same, bit for bit."""
    p = {"small": inputs.plain_small(seed=71),
         "extreme_2e22": inputs.extreme_undersampling(0.08, d=9, seed=72, log2n=22)}.get(
        case, inputs.make_problem(50000, 5000, 7, 1000, 73))
    kw = dict(count=dict(score_mode=ccs.SCORE_COUNT, alpha=3), shifted=dict(shifted=True),
              ordered=dict(debug_flags=2)).get(case, {})
    okw = {k: v for k, v in kw.items() if k != "debug_flags"}
    if "score_mode" in okw:
        okw["score_mode"] = orc.SCORE_COUNT
    csc, ptr, cols, y = device_problem(ccs, p)
    A, y_ref = oracle_problem(orc, p)
    ref = orc.parallel_l0(A, p.m, y_ref, **okw)
    g = ccs.decode_parallel_l0(csc, ptr, cols, y,
                               **dict(kw, debug_flags=kw.get("debug_flags", 0) | 64))
    assert_same_decode(g, ref)

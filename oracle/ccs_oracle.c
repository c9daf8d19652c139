/*
 * ccs_oracle.c -- plain, slow, single-threaded CPU oracle for expander
 * l0-decoding (Mendoza-Smith & Tanner, "Expander l0-decoding", 2015).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the benchmark's CPU
 * baseline use it.  It shares no code, header, table or constant generator
 * with the CUDA library; both sides are written independently from the
 * paper and from the published definitions of the two random-number
 * routines named below.
 *
 * Arithmetic: IEEE binary64, round-to-nearest-even, compiled with
 * -ffp-contract=off and without fast-math, one thread.  Each routine
 * follows the paper's definition step by step, with no blocking, fusion
 * or reordering.
 *
 * Readings of points the paper leaves open (each one is restated where it
 * is used):
 *   R1  Score (Alg. 8 has an empty body): the candidate value omega_j of
 *       column j is the most frequent NONZERO value among r restricted to
 *       N(j); ties go to the numerically smallest value.  One omega per
 *       column and iteration.
 *   R2  Score value: the exact l0 decrease of Eq. (15),
 *       ||r||_0 - ||r - omega a_j||_0 = c_omega - c_0 (default), or the
 *       match count c_omega of Alg. 8 (option).  A pair is accepted when
 *       the score is >= alpha (alpha an integer, 2 <= alpha <= d).
 *   R3  "while not converged": stop when ||r||_0 == 0 (converged), when an
 *       iteration accepts nothing (stalled: Parallel-l0 is deterministic,
 *       so nothing would change again) or after max_iter iterations.  In
 *       the shifted variant (Sec. 4.3.1) an iteration that accepts nothing
 *       leaves r as it was but moves the candidate to the next position, so
 *       it counts as an iteration, and the decode has stalled only when d
 *       iterations in a row accepted nothing: every position has then been
 *       tried on the same r, and the cycle would repeat.  The iteration that
 *       completes such a run is not counted, as in the unshifted rule.
 *   R4  Sums: every row sum over A's columns runs in ascending column
 *       order, starts from +0.0 and skips zero entries (which leaves the
 *       result bit-identical); r_i = y_i - s_i is one subtraction.
 *       -0.0 counts as zero everywhere.
 *   R5  Expander (Sec. 1.1, footnote on generation): column j's d rows are
 *       distinct and uniform over the C(m, d) supports, drawn from the
 *       counter-based SplitMix64 stream of column j with Lemire's bounded
 *       draw, repeated rows redrawn, then sorted ascending.
 *   R12 Column scaling for signals that are not dissociated (Sec. 4.3.3):
 *       "scaling each column by i.i.d. random numbers from a continuous
 *       distribution" is one scale s_j per column, uniform on [1, 2) to a
 *       grid of 2^-20 (1 + the top 20 bits of the first draw of column j's
 *       stream, times 2^-20), so that products with small integers and
 *       their sums stay exact.  The scaled matrix A diag(s) measures
 *       y = A (s . x); Parallel-l0 on A and y recovers z = s . x, and
 *       x = z / s.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "ccs_oracle.h"

/* ------------------------------------------------------------------ */
/* Random numbers                                                      */
/* ------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): a Weyl sequence with
 * increment 0x9e3779b97f4a7c15 followed by the variant-13 finaliser. */
static uint64_t sm64_finalise(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

uint64_t oracle_splitmix64_next(uint64_t *state)
{
    *state += 0x9e3779b97f4a7c15ULL;
    return sm64_finalise(*state);
}

/* Column j's stream starts at seed + (j + 1) * 0xd1b54a32d192ed03 (mod 2^64);
 * its t-th draw (t = 0, 1, ...) is the t-th output of SplitMix64 from there. */
static uint64_t column_stream_start(uint64_t seed, int64_t j)
{
    return seed + (uint64_t)(j + 1) * 0xd1b54a32d192ed03ULL;
}

/* Lemire, "Fast random integer generation in an interval" (ACM TOMACS 2019):
 * multiply a 64-bit draw by the range, keep the high word, and redraw when
 * the low word falls below 2^64 mod range. */
static uint32_t bounded_draw(uint64_t *state, uint32_t range)
{
    uint64_t x = oracle_splitmix64_next(state);
    unsigned __int128 prod = (unsigned __int128)x * range;
    uint64_t low = (uint64_t)prod;
    if (low < range) {
        uint64_t threshold = (0ULL - (uint64_t)range) % range;
        while (low < threshold) {
            x = oracle_splitmix64_next(state);
            prod = (unsigned __int128)x * range;
            low = (uint64_t)prod;
        }
    }
    return (uint32_t)(prod >> 64);
}

/* ------------------------------------------------------------------ */
/* Expander matrix (Defs. 2-3, Sec. 2.2)                               */
/* ------------------------------------------------------------------ */

int oracle_make_expander(int32_t n, int32_t m, int32_t d, uint64_t seed,
                         int32_t *csc_rows)
{
    if (n < 1 || m < 1 || d < 1 || d > m || !csc_rows) return -1;
    for (int64_t j = 0; j < n; ++j) {
        int32_t *col = csc_rows + j * d;
        uint64_t state = column_stream_start(seed, j);
        int got = 0;
        while (got < d) {
            int32_t row = (int32_t)bounded_draw(&state, (uint32_t)m);
            int seen = 0;
            for (int t = 0; t < got; ++t)
                if (col[t] == row) seen = 1;
            if (!seen) col[got++] = row;
        }
        /* insertion sort, ascending */
        for (int a = 1; a < d; ++a) {
            int32_t v = col[a];
            int b = a - 1;
            while (b >= 0 && col[b] > v) { col[b + 1] = col[b]; --b; }
            col[b + 1] = v;
        }
    }
    return 0;
}

/* Column scales (reading R12): s_j = 1 + (first draw of column j's stream
 * >> 44) * 2^-20. */
int oracle_column_scales(int32_t n, uint64_t seed, double *s)
{
    if (n < 1 || !s) return -1;
    for (int64_t j = 0; j < n; ++j) {
        uint64_t state = column_stream_start(seed, j);
        const uint64_t k = oracle_splitmix64_next(&state) >> 44;
        s[j] = 1.0 + (double)k / 1048576.0;
    }
    return 0;
}

/* N(i) for every row i: the transpose of the CSC, columns ascending. */
int oracle_transpose(int32_t n, int32_t m, int32_t d, const int32_t *csc_rows,
                     int64_t *csr_ptr, int32_t *csr_cols)
{
    if (n < 1 || m < 1 || d < 1) return -1;
    int64_t *fill = (int64_t *)calloc((size_t)m, sizeof(int64_t));
    if (!fill) return -2;
    for (int64_t i = 0; i <= m; ++i) csr_ptr[i] = 0;
    for (int64_t e = 0; e < (int64_t)n * d; ++e) {
        int32_t i = csc_rows[e];
        if (i < 0 || i >= m) { free(fill); return -1; }
        csr_ptr[i + 1] += 1;
    }
    for (int64_t i = 0; i < m; ++i) csr_ptr[i + 1] += csr_ptr[i];
    /* visiting columns in ascending order keeps each row's list ascending */
    for (int64_t j = 0; j < n; ++j)
        for (int t = 0; t < d; ++t) {
            int32_t i = csc_rows[j * d + t];
            csr_cols[csr_ptr[i] + fill[i]] = (int32_t)j;
            fill[i] += 1;
        }
    free(fill);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Row sums (R4)                                                       */
/* ------------------------------------------------------------------ */

static double row_sum(const int64_t *csr_ptr, const int32_t *csr_cols,
                      const double *v, int64_t i)
{
    double s = +0.0;
    for (int64_t p = csr_ptr[i]; p < csr_ptr[i + 1]; ++p) {
        double vj = v[csr_cols[p]];
        if (vj != 0.0) s = s + vj;
    }
    return s;
}

/* y = A x (problem statement, Sec. 1): y_i = sum over j in N(i), ascending. */
int oracle_measure(int32_t m, const int64_t *csr_ptr, const int32_t *csr_cols,
                   const double *x, double *y)
{
    for (int64_t i = 0; i < m; ++i) y[i] = row_sum(csr_ptr, csr_cols, x, i);
    return 0;
}

/* y = A diag(s) x (reading R12): y_i = ordered sum over j in N(i) of the
 * nonzero products s_j * x_j (each product rounded once), from +0.0. */
int oracle_measure_scaled(int32_t m, const int64_t *csr_ptr, const int32_t *csr_cols,
                          const double *s, const double *x, double *y)
{
    for (int64_t i = 0; i < m; ++i) {
        double acc = +0.0;
        for (int64_t p = csr_ptr[i]; p < csr_ptr[i + 1]; ++p) {
            const int32_t j = csr_cols[p];
            const double v = s[j] * x[j];
            if (v != 0.0) acc = acc + v;
        }
        y[i] = acc;
    }
    return 0;
}

/* x_j = z_j / s_j: the signal from the decode z of A diag(s)'s measurement. */
int oracle_unscale(int32_t n, const double *s, const double *z, double *x)
{
    for (int64_t j = 0; j < n; ++j) x[j] = z[j] / s[j];
    return 0;
}

/* r = y - A x_hat (Alg. 2, last step of the loop body). */
int oracle_residual(int32_t m, const int64_t *csr_ptr, const int32_t *csr_cols,
                    const double *y, const double *x_hat, double *r)
{
    for (int64_t i = 0; i < m; ++i)
        r[i] = y[i] - row_sum(csr_ptr, csr_cols, x_hat, i);
    return 0;
}

int64_t oracle_l0(int32_t m, const double *r)
{
    int64_t c = 0;
    for (int64_t i = 0; i < m; ++i)
        if (r[i] != 0.0) ++c;
    return c;
}

/* ------------------------------------------------------------------ */
/* Score of one column (Eq. (15), Alg. 8; readings R1, R2)             */
/* ------------------------------------------------------------------ */

/* Returns 1 if the pair (j, omega) is accepted.  Always writes *omega (0.0
 * when no nonzero value is present), *score (c_omega - c_0 or c_omega) and
 * *count (c_omega). */
int oracle_score_column(int32_t d, const int32_t *rows, const double *r,
                        int32_t alpha, int32_t score_mode,
                        double *omega, int32_t *score, int32_t *count)
{
    double v[64];
    int c0 = 0;
    if (d < 1 || d > 64) return -1;
    for (int t = 0; t < d; ++t) {
        v[t] = r[rows[t]];
        if (v[t] == 0.0) ++c0;
    }
    int best = -1, best_count = 0;
    for (int a = 0; a < d; ++a) {
        if (v[a] == 0.0) continue;
        int c = 0;
        for (int b = 0; b < d; ++b)
            if (v[b] == v[a]) ++c;
        if (best < 0 || c > best_count || (c == best_count && v[a] < v[best])) {
            best = a;
            best_count = c;
        }
    }
    if (best < 0) {
        *omega = 0.0;
        *count = 0;
        *score = (score_mode == ORACLE_SCORE_COUNT) ? 0 : -c0;
        return 0;
    }
    *omega = v[best];
    *count = best_count;
    *score = (score_mode == ORACLE_SCORE_COUNT) ? best_count : best_count - c0;
    return *score >= alpha;
}

/* Score of one column in the shifted variant (Sec. 4.3.1, the theorem on
 * shifted Parallel-l0): the only candidate is omega = the value of r at the
 * pos-th row of N(j) (rows ascending, pos counted from 0; reading R11); its
 * count c_omega = #{t : r_{N(j)_t} = omega}, the score as in the other
 * variant.  A zero candidate is never accepted (adding 0 changes nothing).
 * Writes *omega, *score, *count as oracle_score_column. */
int oracle_score_column_shifted(int32_t d, const int32_t *rows, const double *r,
                                int32_t pos, int32_t alpha, int32_t score_mode,
                                double *omega, int32_t *score, int32_t *count)
{
    if (d < 1 || d > 64 || pos < 0 || pos >= d) return -1;
    const double w = r[rows[pos]];
    int c0 = 0, c = 0;
    for (int t = 0; t < d; ++t) {
        const double v = r[rows[t]];
        if (v == 0.0) ++c0;
        if (v == w) ++c;
    }
    if (w == 0.0) {
        *omega = 0.0;
        *count = 0;
        *score = (score_mode == ORACLE_SCORE_COUNT) ? 0 : -c0;
        return 0;
    }
    *omega = w;
    *count = c;
    *score = (score_mode == ORACLE_SCORE_COUNT) ? c : c - c0;
    return *score >= alpha;
}

/* One score pass over all columns, all reading the same r.  shift_pos < 0:
 * the mode of the nonzero values (Alg. 2); else the shifted candidate at
 * that position. */
int64_t oracle_score_all(int32_t n, int32_t d, const int32_t *csc_rows,
                         const double *r, int32_t alpha, int32_t score_mode,
                         int32_t shift_pos, uint8_t *accept, double *omega,
                         int32_t *score)
{
    int64_t accepted = 0;
    for (int64_t j = 0; j < n; ++j) {
        int32_t cnt;
        int a = (shift_pos < 0)
                    ? oracle_score_column(d, csc_rows + j * d, r, alpha, score_mode,
                                          &omega[j], &score[j], &cnt)
                    : oracle_score_column_shifted(d, csc_rows + j * d, r, shift_pos,
                                                  alpha, score_mode, &omega[j],
                                                  &score[j], &cnt);
        accept[j] = (uint8_t)a;
        accepted += a;
    }
    return accepted;
}

/* ------------------------------------------------------------------ */
/* Parallel-l0 (Alg. 2; reading R3 for the stopping rule)              */
/* ------------------------------------------------------------------ */

static int check_params(int32_t d, int32_t alpha, int32_t max_iter,
                        int32_t score_mode)
{
    if (d < 1 || d > 64) return -1;
    if (alpha < 1 || max_iter < 0) return -1;
    if (score_mode != ORACLE_SCORE_L0_DECREASE && score_mode != ORACLE_SCORE_COUNT)
        return -1;
    return 0;
}

/* shifted != 0: the shifted variant, candidate position = iteration mod d. */
int oracle_parallel_l0(int32_t n, int32_t m, int32_t d, const int32_t *csc_rows,
                       const double *y, int32_t alpha, int32_t max_iter,
                       int32_t score_mode, int32_t shifted, double *x_hat, double *r,
                       int64_t *r0_hist, oracle_trace_fn trace, void *trace_ctx,
                       oracle_outcome *out)
{
    if (check_params(d, alpha, max_iter, score_mode)) return -1;
    int64_t *csr_ptr = (int64_t *)malloc(sizeof(int64_t) * ((size_t)m + 1));
    int32_t *csr_cols = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * d);
    uint8_t *accept = (uint8_t *)malloc((size_t)n);
    double *omega = (double *)malloc(sizeof(double) * (size_t)n);
    int32_t *score = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!csr_ptr || !csr_cols || !accept || !omega || !score) {
        free(csr_ptr); free(csr_cols); free(accept); free(omega); free(score);
        return -2;
    }
    int rc = oracle_transpose(n, m, d, csc_rows, csr_ptr, csr_cols);
    if (rc) goto done;

    /* x_hat <- 0, r <- y */
    for (int64_t j = 0; j < n; ++j) x_hat[j] = +0.0;
    for (int64_t i = 0; i < m; ++i) r[i] = y[i];
    int64_t r0 = oracle_l0(m, r);
    int32_t it = 0;
    if (r0_hist) r0_hist[0] = r0;
    int32_t status;
    /* R3: iterations in a row that accepted nothing; the decode stalls at 1
     * (unshifted) or d (shifted: one try of every position on the same r) */
    const int32_t stall_run = shifted ? d : 1;
    int32_t empty_run = 0;
    for (;;) {
        if (r0 == 0) { status = ORACLE_CONVERGED; break; }
        if (it == max_iter) { status = ORACLE_MAX_ITER; break; }
        /* T <- {(j, omega_j) : ||r||_0 - ||r - omega_j a_j||_0 >= alpha} */
        int64_t accepted = oracle_score_all(n, d, csc_rows, r, alpha, score_mode,
                                            shifted ? it % d : -1, accept, omega, score);
        empty_run = (accepted == 0) ? empty_run + 1 : 0;
        if (empty_run == stall_run) { status = ORACLE_STALLED; break; }
        if (trace) trace(trace_ctx, it, n, accept, omega);
        if (accepted == 0) {
            /* shifted: r is unchanged, the next iteration tries the next position */
            it += 1;
            if (r0_hist) r0_hist[it] = r0;
            continue;
        }
        /* for (j, omega_j) in T: x_hat_j <- x_hat_j + omega_j */
        for (int64_t j = 0; j < n; ++j)
            if (accept[j]) x_hat[j] = x_hat[j] + omega[j];
        /* r <- y - A x_hat */
        oracle_residual(m, csr_ptr, csr_cols, y, x_hat, r);
        r0 = oracle_l0(m, r);
        it += 1;
        if (r0_hist) r0_hist[it] = r0;
    }
    out->status = status;
    out->iterations = it;
    out->r0_final = r0;
done:
    free(csr_ptr); free(csr_cols); free(accept); free(omega); free(score);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Serial-l0 (Alg. 1)                                                  */
/* ------------------------------------------------------------------ */

/* One sweep visits j = 0..n-1 in order; after each accepted column the rows
 * of N(j) are recomputed from y and x_hat (the only rows that change), which
 * equals "r <- y - A x_hat" of Alg. 1.  One sweep counts as one iteration
 * (the normalisation by n of Sec. 5). */
int oracle_serial_l0(int32_t n, int32_t m, int32_t d, const int32_t *csc_rows,
                     const double *y, int32_t alpha, int32_t max_iter,
                     int32_t score_mode, int32_t shifted, double *x_hat, double *r,
                     int64_t *r0_hist, oracle_outcome *out)
{
    if (check_params(d, alpha, max_iter, score_mode)) return -1;
    int64_t *csr_ptr = (int64_t *)malloc(sizeof(int64_t) * ((size_t)m + 1));
    int32_t *csr_cols = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * d);
    if (!csr_ptr || !csr_cols) { free(csr_ptr); free(csr_cols); return -2; }
    int rc = oracle_transpose(n, m, d, csc_rows, csr_ptr, csr_cols);
    if (rc) { free(csr_ptr); free(csr_cols); return rc; }

    for (int64_t j = 0; j < n; ++j) x_hat[j] = +0.0;
    for (int64_t i = 0; i < m; ++i) r[i] = y[i];
    int64_t r0 = oracle_l0(m, r);
    int32_t it = 0;
    if (r0_hist) r0_hist[0] = r0;
    int32_t status;
    /* R3, as in Parallel-l0: a sweep that accepts nothing stalls the
     * unshifted decode; the shifted one stalls after d such sweeps in a row */
    const int32_t stall_run = shifted ? d : 1;
    int32_t empty_run = 0;
    for (;;) {
        if (r0 == 0) { status = ORACLE_CONVERGED; break; }
        if (it == max_iter) { status = ORACLE_MAX_ITER; break; }
        int64_t accepted = 0;
        for (int64_t j = 0; j < n; ++j) {
            const int32_t *rows = csc_rows + j * d;
            double omega;
            int32_t score, cnt;
            const int a = shifted ? oracle_score_column_shifted(d, rows, r, it % d, alpha,
                                                                score_mode, &omega, &score,
                                                                &cnt)
                                  : oracle_score_column(d, rows, r, alpha, score_mode,
                                                        &omega, &score, &cnt);
            if (!a) continue;
            x_hat[j] = x_hat[j] + omega;
            for (int t = 0; t < d; ++t) {
                int64_t i = rows[t];
                int was = (r[i] != 0.0);
                r[i] = y[i] - row_sum(csr_ptr, csr_cols, x_hat, i);
                r0 += (r[i] != 0.0) - was;
            }
            ++accepted;
        }
        empty_run = (accepted == 0) ? empty_run + 1 : 0;
        if (empty_run == stall_run) { status = ORACLE_STALLED; break; }
        it += 1;
        if (r0_hist) r0_hist[it] = r0;
    }
    out->status = status;
    out->iterations = it;
    out->r0_final = r0;
    free(csr_ptr); free(csr_cols);
    return 0;
}

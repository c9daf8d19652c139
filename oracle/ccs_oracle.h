/*
 * ccs_oracle.h -- declarations of the CPU oracle (test infrastructure only;
 * see ccs_oracle.c).  Independent of the CUDA library's header.
 */
#ifndef CCS_ORACLE_H
#define CCS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_SCORE_L0_DECREASE = 0, ORACLE_SCORE_COUNT = 1 };
enum { ORACLE_CONVERGED = 0, ORACLE_STALLED = 1, ORACLE_MAX_ITER = 2 };

typedef struct {
    int32_t status;
    int32_t iterations;
    int64_t r0_final;
} oracle_outcome;

/* Called once per Parallel-l0 iteration with the accepted set T (before the
 * update is applied). */
typedef void (*oracle_trace_fn)(void *ctx, int32_t iteration, int32_t n,
                                const uint8_t *accept, const double *omega);

uint64_t oracle_splitmix64_next(uint64_t *state);
int oracle_make_expander(int32_t n, int32_t m, int32_t d, uint64_t seed,
                         int32_t *csc_rows);
int oracle_column_scales(int32_t n, uint64_t seed, double *s);
int oracle_measure_scaled(int32_t m, const int64_t *csr_ptr, const int32_t *csr_cols,
                          const double *s, const double *x, double *y);
int oracle_unscale(int32_t n, const double *s, const double *z, double *x);
int oracle_transpose(int32_t n, int32_t m, int32_t d, const int32_t *csc_rows,
                     int64_t *csr_ptr, int32_t *csr_cols);
int oracle_measure(int32_t m, const int64_t *csr_ptr, const int32_t *csr_cols,
                   const double *x, double *y);
int oracle_residual(int32_t m, const int64_t *csr_ptr, const int32_t *csr_cols,
                    const double *y, const double *x_hat, double *r);
int64_t oracle_l0(int32_t m, const double *r);
int oracle_score_column(int32_t d, const int32_t *rows, const double *r,
                        int32_t alpha, int32_t score_mode, double *omega,
                        int32_t *score, int32_t *count);
int oracle_score_column_shifted(int32_t d, const int32_t *rows, const double *r,
                                int32_t pos, int32_t alpha, int32_t score_mode,
                                double *omega, int32_t *score, int32_t *count);
int64_t oracle_score_all(int32_t n, int32_t d, const int32_t *csc_rows,
                         const double *r, int32_t alpha, int32_t score_mode,
                         int32_t shift_pos, uint8_t *accept, double *omega,
                         int32_t *score);
int oracle_parallel_l0(int32_t n, int32_t m, int32_t d, const int32_t *csc_rows,
                       const double *y, int32_t alpha, int32_t max_iter,
                       int32_t score_mode, int32_t shifted, double *x_hat, double *r,
                       int64_t *r0_hist, oracle_trace_fn trace, void *trace_ctx,
                       oracle_outcome *out);
int oracle_serial_l0(int32_t n, int32_t m, int32_t d, const int32_t *csc_rows,
                     const double *y, int32_t alpha, int32_t max_iter,
                     int32_t score_mode, int32_t shifted, double *x_hat, double *r,
                     int64_t *r0_hist, oracle_outcome *out);

#ifdef __cplusplus
}
#endif
#endif

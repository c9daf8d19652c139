/*
 * ccs.h -- C ABI of libccs, a GB300 (sm_103a) implementation of the
 * Parallel-l0 expander decoder of Mendoza-Smith & Tanner, "Expander
 * l0-decoding" (2015).
 *
 * Problem (Sec. 1): recover a k-sparse x in R^n from y = A x in R^m, where A
 * is the 0/1 adjacency matrix of a left d-regular bipartite expander
 * (Defs. 2-3, Sec. 2.2): column j has ones exactly in the d rows N(j).
 *
 * Conventions shared by every entry point:
 *  - Array arguments are DEVICE pointers owned by the caller (for example
 *    PyTorch tensors' data_ptr()).  The library never frees or keeps them.
 *  - Scratch comes from a caller-owned device workspace of at least the size
 *    the matching *_workspace_size() call reports; no call on the decode path
 *    allocates device memory.  A workspace serves one call at a time.
 *  - Work is issued on the caller's stream (a cudaStream_t; NULL is the
 *    legacy default stream).  Calls that report a result to the host say
 *    so and synchronise that stream before returning.
 *  - Every call returns a status code (CCS_OK or a CCS_E* error); nothing
 *    is thrown across the ABI.  ccs_last_error() describes the last failure
 *    of the calling thread.  The decode outcome (converged / stalled /
 *    iteration cap) is a field of ccs_result, not an error.
 *  - Matrix layout: CSC row indices csc_rows[n*d], int32; column j's d
 *    distinct rows sit at [j*d, (j+1)*d), ascending.  CSR (the transpose,
 *    N(i) for every row i): csr_ptr[m+1] int64 offsets, csr_cols[n*d] int32,
 *    columns ascending within each row.
 *  - Values are IEEE binary64.  Every sum over a row runs in ascending
 *    column order from +0.0, skipping zero entries; -0.0 counts as zero.
 *    Inputs must be finite.
 *  - Limits: 1 <= d <= 16, d <= m, n*d < 2^31.
 *  - Alignment: csc_rows on 16 bytes (it is bulk-copied), binary64 and
 *    int64 arrays on 8, csr_cols on 4, workspaces and the server pool on
 *    256.  Fresh cudaMalloc / PyTorch allocations meet all of these; a
 *    pointer that does not is refused with CCS_EINVAL before any device
 *    work (on the device it would fault).
 */
#ifndef CCS_H
#define CCS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define CCS_API __attribute__((visibility("default")))
#else
#define CCS_API
#endif

/* Same object as cudaStream_t, declared here so that this header does not
 * need the CUDA headers. */
typedef struct CUstream_st *ccs_stream_t;

/* ---- status codes ------------------------------------------------------ */
enum {
    CCS_OK = 0,
    CCS_EINVAL = 1,    /* bad argument or size outside the limits above      */
    CCS_ENOMEM = 2,    /* workspace smaller than *_workspace_size()          */
    CCS_ECUDA = 3,     /* a CUDA runtime call failed                         */
    CCS_ETIMEOUT = 4,  /* a bounded device wait ran out (watchdog)           */
    CCS_EBUDGET = 5,   /* serving: request does not fit the memory budget    */
    CCS_EBUSY = 6      /* serving: no free slot / ticket not finished        */
};

/* ---- decode outcome (ccs_result.status) -------------------------------- */
enum {
    CCS_CONVERGED = 0, /* ||r||_0 == 0, i.e. y == A x_hat                     */
    CCS_STALLED = 1,   /* an iteration accepted no pair: a fixed point       */
    CCS_MAX_ITER = 2   /* params.max_iter iterations done                    */
};

/* ---- score (selection rule) -------------------------------------------- */
enum {
    /* Eq. (15): the l0 decrease ||r||_0 - ||r - omega a_j||_0, which for a
     * 0/1 column with distinct rows equals c_omega - c_0 (matches of omega
     * minus zeros among r_N(j)).  Default. */
    CCS_SCORE_L0_DECREASE = 0,
    /* Alg. 8 (and the rule of ER / LDDSR, Sec. 3): the match count c_omega. */
    CCS_SCORE_COUNT = 1
};

/* ---- engines ------------------------------------------------------------ */
enum {
    CCS_ENGINE_AUTO = 0,       /* library's choice                           */
    CCS_ENGINE_HOST_LOOP = 1,  /* one launch per phase, host checks the stop
                                  rule after every iteration                 */
    CCS_ENGINE_PERSISTENT = 3  /* one cooperative launch runs every
                                  iteration; grid barriers between phases,
                                  each wait bounded by watchdog_ms           */
};

typedef struct {
    int32_t alpha;        /* accept when score >= alpha; 2 <= alpha <= d.
                             The paper's real alpha in (1, d] is ceil(alpha).
                             Default 2 (Sec. 5).                              */
    int32_t max_iter;     /* iteration cap, >= 0; default 100                 */
    int32_t score_mode;   /* CCS_SCORE_*; default CCS_SCORE_L0_DECREASE       */
    int32_t engine;       /* CCS_ENGINE_*; default CCS_ENGINE_AUTO            */
    int32_t watchdog_ms;  /* bound on every device-side wait; 0 = 2000 ms     */
    int32_t debug_flags;  /* test hooks, 0 in normal use.  Bit 0 (persistent
                             engine): CTA 0 skips its arrival at the first
                             score barrier, so every CTA's bounded wait runs
                             out and the call returns CCS_ETIMEOUT.  Bit 1:
                             the persistent engine keeps the residual by
                             ordered row sums from the first iteration
                             instead of by exact atomic updates.  Bit 2: the
                             test that certifies those updates exact is
                             treated as failing from iteration 2, so the
                             decode switches residual mode mid-way.  Bits
                             3-5 (persistent engine, one problem per
                             launch) steer the row-driven score phase: bit 3
                             scores its candidates one by one instead of
                             queueing them, bit 4 takes it whenever its row
                             list fits instead of only once ||r||_0 <= m/64
                             on a CSC of at least 2^26 entries, bit 5 never
                             takes it.  Bit 6: the column stream scores
                             every candidate where it finds it instead of
                             queueing it.  Results are the same for every
                             setting of bits 1-6.                            */
    int32_t schedule;     /* persistent-engine launch shape, 0..127.
                             Bits 0-1, the thread shape: 0 = library's
                             choice (1 when d <= 8, else 2); 1 = 1024
                             threads a CTA, one 32-column tile per warp and
                             chunk (d <= 8 only); 2 = 512 threads, two
                             tiles per warp and chunk; 3 = 768 threads, one
                             tile per warp and chunk (d <= 8 only).
                             Bits 2-4: the CSC stage ring's depth, 0 = as
                             many stages as shared memory holds (at most
                             6), else 2..6 at most.  Bits 5-6: the queue of
                             candidate columns, 0 = as long as shared
                             memory allows (at most 2048 a CTA), 1 = 256
                             entries, 2 = 1024.  0 as a whole: the shape
                             ccs_autotune recorded for this class of launch
                             on this device, else the library's choice.   */
    int32_t shifted;      /* 0: Alg. 2, each column's candidate is the mode of
                             its nonzero residual values.  1: the shifted
                             variant of Sec. 4.3.1: at iteration l the only
                             candidate is the value of r at the (l mod d)-th
                             row of the column (rows ascending, counted from
                             0); O(d) per column for any alpha.  Persistent
                             engine only.  Default 0.                        */
} ccs_params;

typedef struct {
    int32_t status;       /* CCS_CONVERGED / CCS_STALLED / CCS_MAX_ITER        */
    int32_t iterations;   /* completed iterations (each one: score all
                             columns, apply, recompute r)                    */
    int64_t r0_final;     /* ||r||_0 at exit                                   */
    int32_t error;        /* CCS_OK, or the CCS_E* code that ended this
                             problem early (e.g. CCS_ETIMEOUT)               */
    int32_t row_driven;   /* iterations whose score phase was row-driven:
                             once ||r||_0 <= m/64 on a CSC too large for L2
                             (n d >= 2^26), the persistent engine (one
                             problem per launch) finds the columns that can
                             still be accepted from the CSR rows of the
                             nonzero r_i instead of streaming every column
                             (same results)                                  */
    int64_t row_entries;  /* CSR entries those score phases read            */
    int32_t residual_form;/* how r = y - A x_hat was kept when the decode
                             ended (same results either way):
                             CCS_RESIDUAL_EXACT or CCS_RESIDUAL_ORDERED      */
    int32_t reserved;
} ccs_result;

/* ccs_result.residual_form.  Alg. 2 recomputes r_i = y_i minus the ordered
 * sum of the row's nonzero x_hat_j.  While every value of the decode lies on
 * the grid of y and far enough below 2^53 grid steps, binary64 additions are
 * exact and the persistent engine keeps r by subtracting each accepted omega
 * instead (EXACT; the bound is checked before every iteration).  Once it
 * fails, the decode recomputes every touched row by its ordered sum for the
 * rest of the decode (ORDERED; the host-driven engine always does). */
enum { CCS_RESIDUAL_EXACT = 0, CCS_RESIDUAL_ORDERED = 1 };

/* One problem of a batch: sizes and caller-owned device arrays. */
typedef struct {
    int32_t n, m, d, reserved;
    const int32_t *csc_rows;  /* n*d                                         */
    const int64_t *csr_ptr;   /* m+1                                         */
    const int32_t *csr_cols;  /* n*d                                         */
    const double *y;          /* m                                           */
    double *x_hat;            /* out, n                                      */
    double *r;                /* out, m: y - A x_hat at exit                 */
    int64_t *r0_hist;         /* optional out, max_iter+1 entries (NULL: off) */
} ccs_problem;

/* Workspace sizes (bytes) for the calls below. */
enum { CCS_OP_MAKE_EXPANDER = 0, CCS_OP_DECODE = 1 };

/* Fills *p with the defaults listed in ccs_params. */
CCS_API void ccs_params_init(ccs_params *p);

/* Human-readable name of a status code (static string). */
CCS_API const char *ccs_status_string(int status);

/* Description of the calling thread's last failed call (static per thread). */
CCS_API const char *ccs_last_error(void);

/* Library version, major*10000 + minor*100 + patch. */
CCS_API int ccs_version(void);

/* Bytes of workspace that ccs_make_expander (op = CCS_OP_MAKE_EXPANDER) or
 * ccs_decode_parallel_l0 (op = CCS_OP_DECODE) needs for these sizes;
 * 0 if the sizes are invalid. */
CCS_API size_t ccs_workspace_size(int32_t op, int32_t n, int32_t m, int32_t d);

/* Bytes of workspace that ccs_decode_batch needs for these problems. */
CCS_API size_t ccs_batch_workspace_size(const ccs_problem *probs, int32_t count);

/*
 * ccs_make_expander -- draw a random left d-regular expander and its
 * transpose (Sec. 1.1 footnote: columns iid, each column's support uniform
 * over the C(m, d) subsets of size d; Table 1: O(dn) generation).
 *
 * Column j takes the SplitMix64 stream (Steele, Lea & Flood 2014) that
 * starts at seed + (j+1) * 0xd1b54a32d192ed03 mod 2^64, maps each draw to a
 * row with Lemire's bounded method (ACM TOMACS 2019), redraws repeated rows
 * and sorts its d rows.  The result depends only on (n, m, d, seed).
 *
 * out: csc_rows[n*d], csr_ptr[m+1], csr_cols[n*d] (device).
 * Synchronises the stream.  CCS_EINVAL if the sizes break the limits or a
 * row ends up with more than 32768 columns (rows are sorted on chip).
 */
CCS_API int ccs_make_expander(int32_t n, int32_t m, int32_t d, uint64_t seed,
                      int32_t *csc_rows, int64_t *csr_ptr, int32_t *csr_cols,
                      void *ws, size_t ws_bytes, ccs_stream_t stream);

/*
 * ccs_measure -- y = A x (Sec. 1, problem statement): y_i is the sum of
 * x_j over j in N(i) in ascending j, from +0.0, zero x_j skipped.
 * in: csr_ptr, csr_cols, x[n]; out: y[m] (device).  Asynchronous.
 */
CCS_API int ccs_measure(int32_t n, int32_t m, int32_t d, const int64_t *csr_ptr,
                const int32_t *csr_cols, const double *x, double *y,
                ccs_stream_t stream);

/* ---- column-scaled A for signals that are not dissociated (Sec. 4.3.3) -------
 *
 * When x has equal nonzero values (binary or integer signals), scaling each
 * column of A by an i.i.d. continuous random number makes the measured
 * values identifiable again.  Here A diag(s) has one scale s_j per column.
 *
 * ccs_column_scales writes s[0..n): s_j = 1 + k_j 2^-20 with k_j the top 20
 *   bits of the first draw of column j's SplitMix64 stream from `seed` (the
 *   same stream rule as ccs_make_expander), so s_j is uniform on [1, 2) on a
 *   2^-20 grid and products with small integers stay exact.  Device output;
 *   CCS_EINVAL when n < 1 or s is null.
 * ccs_measure_scaled writes y = A diag(s) x: y_i = ordered sum over the
 *   row's columns j (ascending) of the nonzero products s_j * x_j, each
 *   rounded once, from +0.0.  Arguments and errors as ccs_measure.
 * ccs_unscale writes x_j = z_j / s_j (correctly rounded): decoding y with
 *   any ccs_decode_* entry point on the unscaled A recovers z = s . x, and
 *   this returns x.  In-place use (x == z) is allowed.
 * All three are stream-ordered on `stream` and allocate nothing.          */
CCS_API int ccs_column_scales(int32_t n, uint64_t seed, double *s, ccs_stream_t stream);
CCS_API int ccs_measure_scaled(int32_t n, int32_t m, int32_t d, const int64_t *csr_ptr,
                               const int32_t *csr_cols, const double *s, const double *x,
                               double *y, ccs_stream_t stream);
CCS_API int ccs_unscale(int32_t n, const double *s, const double *z, double *x,
                        ccs_stream_t stream);

/*
 * ccs_decode_parallel_l0 -- Parallel-l0 (Alg. 2).
 *
 *   x_hat <- 0, r <- y
 *   while not converged:
 *     for every column j, reading the same r: omega_j = the most frequent
 *       nonzero value of r on N(j) (ties: the smallest), accepted when its
 *       score (Eq. (15) or Alg. 8, see score_mode) is >= alpha
 *     x_hat_j <- x_hat_j + omega_j for all accepted j at once
 *     r <- y - A x_hat, ||r||_0
 *
 * "Converged" is read as: stop when ||r||_0 == 0 (CCS_CONVERGED), when no
 * pair is accepted (CCS_STALLED; the iteration is deterministic so nothing
 * would change again) or after max_iter iterations (CCS_MAX_ITER).
 *
 * in:  csc_rows, csr_ptr, csr_cols, y (device)
 * out: x_hat[n], r[m] (device); r0_hist[max_iter+1] (device, optional:
 *      entry t = ||r||_0 after t iterations, entries past the last
 *      iteration untouched); *out (host memory).
 * p may be NULL (defaults).  Blocks until the decode has finished.
 * Errors: CCS_EINVAL (sizes, alpha outside [2, d], bad params),
 * CCS_ENOMEM (ws_bytes too small), CCS_ECUDA, CCS_ETIMEOUT.
 */
CCS_API int ccs_decode_parallel_l0(int32_t n, int32_t m, int32_t d,
                           const int32_t *csc_rows, const int64_t *csr_ptr,
                           const int32_t *csr_cols, const double *y,
                           double *x_hat, double *r, int64_t *r0_hist,
                           const ccs_params *p, ccs_result *out,
                           void *ws, size_t ws_bytes, ccs_stream_t stream);

/*
 * ccs_decode_parallel_l0_async -- the same decode, enqueued on the stream
 * without waiting: the persistent engine writes the ccs_result into DEVICE
 * memory out_dev when the decode ends (error = CCS_ETIMEOUT if a bounded
 * wait ran out).  The host-driven engine is not available here (CCS_EINVAL).
 * The workspace and outputs must stay untouched until the stream reaches
 * that point.  Argument checks as for ccs_decode_parallel_l0; CUDA errors of
 * the launch itself are returned, later ones surface on the stream.
 */
CCS_API int ccs_decode_parallel_l0_async(int32_t n, int32_t m, int32_t d,
                                         const int32_t *csc_rows, const int64_t *csr_ptr,
                                         const int32_t *csr_cols, const double *y,
                                         double *x_hat, double *r, int64_t *r0_hist,
                                         const ccs_params *p, ccs_result *out_dev,
                                         void *ws, size_t ws_bytes, ccs_stream_t stream);

/*
 * ccs_decode_batch -- Parallel-l0 on `count` independent problems of any
 * sizes in persistent cooperative launches (the iteration loop runs on the
 * device; each problem stops on its own rule and drops out of later
 * phases).  Problems of one class (d <= 8 or d > 8; fingerprints of r in
 * shared memory or not) share a launch; when a batch holds several classes,
 * each class's launch runs a few iterations, then one launch over the whole
 * batch continues the problems still running.  Per problem, the results are
 * bit-identical to ccs_decode_parallel_l0 on that problem alone.
 *
 * probs: host array of `count` descriptors (device pointers inside);
 * out: host array of `count` results.  Blocks until every problem has
 * finished.  Errors as for ccs_decode_parallel_l0.
 */
CCS_API int ccs_decode_batch(const ccs_problem *probs, int32_t count,
                     const ccs_params *p, ccs_result *out,
                     void *ws, size_t ws_bytes, ccs_stream_t stream);

/* ccs_decode_batch enqueued without waiting; results (count entries) go to
 * DEVICE memory out_dev, as for ccs_decode_parallel_l0_async. */
CCS_API int ccs_decode_batch_async(const ccs_problem *probs, int32_t count,
                                   const ccs_params *p, ccs_result *out_dev,
                                   void *ws, size_t ws_bytes, ccs_stream_t stream);

/* ---- launch-shape autotuner ---------------------------------------------------
 *
 * Not in the paper (its method fixes no launch configuration).  A batched
 * decode goes out as up to four launches, one per class of problem (d <= 8
 * or d > 8; fingerprints of r in shared memory or not).  ccs_autotune
 * decodes `probs` as ccs_decode_batch would, but runs each launch group with
 * every launch shape its kernel instances offer (CTAs of 1024, 768 or 512
 * threads for d <= 8; 512 for d > 8; each with the CSC ring at full depth or
 * capped at 2 or 3 stages, and the candidate queue at full length or capped
 * at 256 entries: 18 shapes for d <= 8, 6 above), twice each, timing the
 * second run with CUDA events on `stream`.  The fastest shape of each group is recorded
 * in a table inside the library, per device and class (largest d of the
 * launch, fingerprint fit); from then on every launch on that device with
 * p->schedule == 0 in that class uses it.  tuned[0..3] receives the shape
 * picked for each group in launch order (0 for groups that do not exist).
 * Arguments, workspace and errors as ccs_decode_batch; the outputs hold the
 * last run's decode (every shape gives the same results).  Blocks the
 * calling thread.  ccs_autotune_reset clears the table.                   */
CCS_API int ccs_autotune(const ccs_problem *probs, int32_t count, const ccs_params *p,
                         void *ws, size_t ws_bytes, ccs_stream_t stream, int32_t *tuned);
CCS_API void ccs_autotune_reset(void);
/* The table's entry for the current device and a class (largest d of a
 * launch, fingerprints of r in shared memory or not): the schedule code, 0
 * when none is recorded. */
CCS_API int ccs_autotune_get(int32_t dmax, int32_t fits, int32_t *schedule);
/* The table on disk: ccs_autotune_save writes every recorded entry of every
 * visible device, one line "gpu dmax fits schedule", the gpu keyed by
 * model (name, SM count, compute capability); ccs_autotune_load installs
 * the entries whose key matches a visible device, so a shape tuned once
 * serves later processes on the same GPU model.  CCS_EINVAL when the file
 * cannot be written or read; malformed lines are skipped. */
CCS_API int ccs_autotune_save(const char *path);
CCS_API int ccs_autotune_load(const char *path);

/* ---- CUDA graph of a batched decode -----------------------------------------
 *
 * ccs_batch_graph_create captures the launches ccs_decode_batch_async makes
 * for these problems (the launch header resets and the persistent kernels)
 * into a CUDA graph; the problem descriptors are uploaded to the workspace
 * once, now.
 * Each ccs_graph_launch replays the whole decode of every problem on the
 * same device arrays and workspace (write new y values in place between
 * replays to decode new measurements), results to DEVICE memory out_dev as
 * for ccs_decode_batch_async.  Replays on one graph must not overlap.  The
 * workspace, arrays and out_dev must outlive the graph.  Synchronous during
 * creation (it uploads and instantiates). */
typedef struct ccs_graph ccs_graph;
CCS_API int ccs_batch_graph_create(const ccs_problem *probs, int32_t count,
                                   const ccs_params *p, ccs_result *out_dev,
                                   void *ws, size_t ws_bytes, ccs_graph **out);
CCS_API int ccs_graph_launch(ccs_graph *g, ccs_stream_t stream);
CCS_API int ccs_graph_destroy(ccs_graph *g);

/* ---- serving: continuous batching -----------------------------------------
 *
 * A decode server with one worker thread.  Requests (ccs_problem: device
 * arrays owned by the caller, kept alive until their result is collected)
 * are queued by ccs_server_submit.  The worker runs engine rounds: one
 * persistent launch over every admitted request, at most iters_per_round
 * iterations of Alg. 2, each request's decode state kept on the device
 * between rounds.  After each round finished requests are retired and
 * pending ones admitted, in arrival order, as long as their state fits the
 * memory pool and a batch slot is free; so requests arriving while others
 * run join them on the GPU.  Every result is bit-identical to
 * ccs_decode_parallel_l0 on the same request.  Not in the paper: a serving
 * layer over its decoder.
 */
typedef struct ccs_server ccs_server;

typedef struct {
    void *pool;               /* caller-owned device memory the server carves
                                 request state and its launch header from    */
    size_t pool_bytes;        /* its size: the HBM budget for request state  */
    int32_t max_batch;        /* most requests in one round, 1..4096         */
    int32_t iters_per_round;  /* iterations per round, >= 1                  */
    ccs_params params;        /* decode parameters of every request          */
} ccs_server_config;

typedef struct {
    ccs_result result;        /* as ccs_decode_parallel_l0 reports it        */
    double submit_s, admit_s, done_s;  /* steady-clock seconds (one origin
                                 per process): queued, admitted, finished    */
    int32_t rounds;           /* engine rounds the request took part in      */
    int32_t reserved;
} ccs_ticket_info;

typedef struct {
    int64_t submitted, admitted, completed, rounds;
    int64_t peak_inflight;    /* most requests in one round                  */
    int64_t peak_bytes;       /* most pool bytes in use by request state     */
    int64_t bytes_in_use, pending, inflight;
    int32_t error;            /* first CCS_E* a round returned, else CCS_OK  */
    int32_t reserved;
} ccs_server_stats;

/* A request whose device memory the server owns (not in the paper).  The
 * caller gives the expander's seed and HOST buffers; at admission the server
 * draws A into the pool from (n, m, d, a_seed) exactly as ccs_make_expander
 * does and copies y from the host, so everything the request keeps on the
 * device -- A as CSC and CSR, y, x_hat, r, the ||r||_0 history and the
 * decode state, ccs_seeded_request_bytes() in all -- comes out of the pool,
 * and the pool bounds the server's HBM.  When the decode ends, x_hat (and
 * r, r0_hist when non-null) are copied to the host buffers before the
 * result is published and the memory returns to the pool.  The host
 * buffers must stay valid, and y unchanged, until the result is collected.
 * Results are bit-identical to ccs_decode_parallel_l0 on the same A and y. */
typedef struct {
    int32_t n, m, d, reserved;
    uint64_t a_seed;          /* seed of A, as for ccs_make_expander         */
    const double *y;          /* HOST, m measurements                        */
    double *x_hat;            /* HOST out, n; optional when the nonzeros are
                                 asked for below                             */
    double *r;                /* HOST out, m: y - A x_hat at exit; optional  */
    int64_t *r0_hist;         /* HOST out, max_iter+1 entries; optional      */
    /* x_hat as its nonzero entries (optional, all three or none): the
     * server lists them on the device and copies back only those.
     * *x_nnz = their number nnz; x_idx / x_val receive min(nnz, x_cap) of
     * them, indices ascending -- all of them when nnz <= x_cap, else an
     * unspecified subset (ask again with x_cap >= nnz).  A decoded
     * k-sparse x_hat moves 16 k bytes instead of 8 n. */
    int64_t *x_idx;           /* HOST out, x_cap entries                     */
    double *x_val;            /* HOST out, x_cap entries                     */
    int64_t x_cap;            /* >= 1 when the nonzeros are asked for        */
    int64_t *x_nnz;           /* HOST out, one entry                         */
} ccs_seeded_request;

/* Pool bytes one seeded request holds while admitted: A, y, x_hat, r, the
 * history, the decode state, the generation workspace, and 8 + 16 x_cap
 * for the nonzero list (x_cap = 0 when the request asks for none).  0 for
 * invalid sizes. */
CCS_API size_t ccs_seeded_request_bytes(int32_t n, int32_t m, int32_t d, int32_t max_iter,
                                        int64_t x_cap);

/* Starts the worker on the current device; work goes to `stream`.
 * CCS_EINVAL for a bad configuration, CCS_EBUDGET if the pool cannot even
 * hold the launch header. */
CCS_API int ccs_server_create(const ccs_server_config *cfg, ccs_stream_t stream,
                              ccs_server **out);
/* Queues a request; *ticket identifies it.  CCS_EBUDGET if its state can
 * never fit the pool, CCS_EINVAL for bad sizes or arrays. */
CCS_API int ccs_server_submit(ccs_server *s, const ccs_problem *req, int64_t *ticket);
/* Queues a seeded request (see ccs_seeded_request).  CCS_EBUDGET if
 * ccs_seeded_request_bytes() can never fit the pool, CCS_EINVAL for bad
 * sizes, a null y, or neither x_hat nor a complete nonzero-list request.  A failure while drawing A or copying data ends
 * the request with that code in its result's error field. */
CCS_API int ccs_server_submit_seeded(ccs_server *s, const ccs_seeded_request *req,
                                     int64_t *ticket);
/* CCS_OK and *info once the request has finished (the ticket is then
 * released); CCS_EBUSY while it is pending or running. */
CCS_API int ccs_server_poll(ccs_server *s, int64_t ticket, ccs_ticket_info *info);
/* As ccs_server_poll, waiting up to timeout_ms for the result. */
CCS_API int ccs_server_wait(ccs_server *s, int64_t ticket, ccs_ticket_info *info,
                            int32_t timeout_ms);
CCS_API int ccs_server_stats_get(ccs_server *s, ccs_server_stats *out);
/* Finishes every queued request, stops the worker, frees the handle.
 * Returns the first error a round reported, else CCS_OK. */
CCS_API int ccs_server_destroy(ccs_server *s);

/*
 * ccs_decode_parallel_l0_noalloc -- ccs_decode_parallel_l0 for callers that
 * cannot allocate device memory when they decode (a memory budget that is
 * already fully reserved, a real-time loop where an allocation and the
 * synchronisation it may bring are not allowed, a host that only hands out
 * pre-registered buffers).  The paper has no counterpart: this is a
 * deployment variant of the same decode, with the same results.
 *
 * The caller passes the inputs and outputs as for ccs_decode_parallel_l0
 * but no workspace: the scratch is one device array of
 * ccs_noalloc_scratch_bytes() bytes (16 MiB) that the library keeps in every
 * GPU that loads it, until the process exits.  Sizes whose workspace
 * (ccs_workspace_size(CCS_OP_DECODE, n, m, d)) exceeds it are rejected with
 * CCS_EINVAL; n = 2^20, m = 2^17, d = 7 fits.  The call allocates nothing:
 * no cudaMalloc, no cudaFree, no allocating library routine.  Its first call
 * on a device looks up that device's address of the array
 * (cudaGetSymbolAddress) and keeps it for the life of the process; make that
 * first call before any stream capture.  A cudaDeviceReset invalidates the
 * kept address, so no call may follow a reset of the device.
 * Every call on a device shares the one array, which keeps the last call's
 * contents (the decode clears what must start at zero), so calls whose
 * work overlaps on the GPU race: issue them one after another on one stream
 * or otherwise order them.  Persistent engine only (CCS_ENGINE_HOST_LOOP is
 * CCS_EINVAL).  Blocks until the decode has finished.
 */
CCS_API int ccs_decode_parallel_l0_noalloc(int32_t n, int32_t m, int32_t d,
                                           const int32_t *csc_rows, const int64_t *csr_ptr,
                                           const int32_t *csr_cols, const double *y,
                                           double *x_hat, double *r, int64_t *r0_hist,
                                           const ccs_params *p, ccs_result *out,
                                           ccs_stream_t stream);

/* Bytes of the static scratch behind ccs_decode_parallel_l0_noalloc. */
CCS_API size_t ccs_noalloc_scratch_bytes(void);

/* ---- measurement hooks ---------------------------------------------------
 * Kernel timing for benchmarks: between ccs_profile_begin() and
 * ccs_profile_end() the library brackets each of its kernel launches with
 * CUDA events on the launching stream and sums the elapsed device time per
 * kernel kind.  Off by default (no events are recorded when off).  Process-
 * wide; not meant to be used from several threads at once. */
enum {
    CCS_K_INIT = 0,        /* x_hat <- 0, r <- y, ||y||_0                   */
    CCS_K_SCORE = 1,       /* score + apply (all columns)                   */
    CCS_K_RESIDUAL = 2,    /* r on touched rows + ||r||_0                    */
    CCS_K_FINISH = 3,      /* stop rule                                      */
    CCS_K_PERSISTENT = 4,  /* whole decode in one cooperative launch; its
                              score and residual phases are also reported
                              under CCS_K_SCORE / CCS_K_RESIDUAL (device
                              timer between grid barriers, one entry per
                              iteration)                                    */
    CCS_K_PHASE_FP = 5,     /* score phase seen from CTA 0: wait for the
                              residual fingerprints                         */
    CCS_K_PHASE_STREAM = 6, /* ... stream of the CSC through the fingerprint
                              filter                                        */
    CCS_K_PHASE_QUEUE = 7,  /* ... exact scoring of the queued candidates    */
    CCS_K_COUNT = 8
};
typedef struct {
    int64_t launches;
    double total_ms;
} ccs_kernel_time;

CCS_API int ccs_profile_begin(void);
/* times: array of CCS_K_COUNT entries (host). */
CCS_API int ccs_profile_end(ccs_kernel_time *times);
/* Phase times of one iteration of the last persistent launch made while
 * profiling (device timer between grid barriers): phase_us[0] score phase,
 * [1] residual phase, [2..4] CTA 0's score sub-phases (fingerprints in,
 * stream, queued candidates; -1 when not recorded).  CCS_EINVAL if that
 * iteration was not recorded. */
CCS_API int ccs_profile_phases(int32_t iteration, double *phase_us);
/* Number of kernels this library has launched since it was loaded. */
CCS_API int64_t ccs_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* CCS_H */

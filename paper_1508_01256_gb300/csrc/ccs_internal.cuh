// ccs_internal.cuh -- device helpers shared by the libccs translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include <vector>

#include "ccs.h"

namespace ccs {

constexpr int kMaxD = 16;           // register-resident gather of d <= 16 values
constexpr int kSlots = 15;          // contributor slots kept per row (+1 count word)
constexpr int kSlotRec = 16;        // ints per row record: count, then kSlots columns
constexpr int kMaxSortRow = 32768;  // longest CSR row sorted on chip
constexpr int kRunning = -1;        // DecodeCtrl::status while iterating

enum ProblemFlags : int {
    kPdUseFp = 1,
    kPdFresh = 2,
};

enum ErrorBits : int {
    kErrWatchdog = 1,
};

// Per-problem decode state kept in the workspace (device memory).
struct alignas(64) DecodeCtrl {
    unsigned long long acc[4];  // accepted pairs, ring indexed by iteration & 3
    long long r0;               // ||r||_0 of the current r (residual phases add
                                // their exact integer change)
    int iteration;              // completed iterations
    int status;                 // kRunning or CCS_CONVERGED / _STALLED / _MAX_ITER
    int error;                  // ErrorBits
    int max_iter;
    // Exactness certificate of the incremental residual (persistent engine):
    int grid_b;                 // 1100 - (exponent of the lowest set bit over the
                                // nonzero y_i); 0 when y == 0
    int deg;                    // largest row degree of A
    unsigned long long ymax;    // bits of max |y_i|
    unsigned long long rmax[2]; // bits of max |r_i| at the start of iteration t
                                // (slot t & 1)
    unsigned long long xmax[2]; // bits of an upper bound of every |x_hat_j| so far
                                // at the start of iteration t (slot t & 1)
    int ordered;                // 1 once the problem runs the ordered residual
    int empty_run[2];           // iterations in a row that accepted nothing, before
                                // iteration t (slot t & 1; persistent engine)
    int row_driven;             // iterations whose score phase went row-driven
    long long row_entries;      // CSR entries those score phases read
};
static_assert(sizeof(DecodeCtrl) == 128, "DecodeCtrl layout");

// Device view of one problem plus its slice of the workspace.
struct ProblemDev {
    int n, m, d;
    int flags;            // kPdUseFp: fingerprints fit shared memory (engine);
                          // kPdFresh: initialise before iterating (resume mode)
    int out_slot;         // index of this problem's entry in the engine's
                          // device-side result array
    const int32_t *csc_rows;
    const int64_t *csr_ptr;
    const int32_t *csr_cols;
    const double *y;
    double *x_hat;
    double *r;
    double *r_next;       // m: r updated in place by the accepted pairs while the
                          // incremental residual is exact (persistent engine)
    int64_t *r0_hist;     // may be null
    DecodeCtrl *ctrl;
    uint8_t *touched;     // m: rows whose sum must be recomputed
    uint8_t *in_slots;    // n: column already entered in its rows' slots
    int32_t *slots;       // m * kSlotRec: per row, one 64-byte record holding the
                          // number of columns entered and (up to kSlots of)
                          // those columns, unordered
    uint8_t *fp;          // m fingerprints of r_i (0 iff r_i == 0): 16-bit when
                          // fp16_for(m), else 8-bit
    uint32_t *hits;       // ceil(n/4) words, one byte per column: the nonzero rows
                          // a row-driven score phase counted for the column
                          // (zero between phases; persistent engine, one problem)
};

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Problems with at most kFp16MaxM rows keep 16-bit residual fingerprints
// (2m bytes, 64 KB at most), the others 8-bit ones.  The width depends on m
// alone, so every launch that reads or writes a problem's fingerprints
// agrees on it (a served problem meets several launch plans).
constexpr int kFp16MaxM = 32768;
__host__ __device__ inline bool fp16_for(int m) { return m <= kFp16MaxM; }
__host__ __device__ inline size_t fp_bytes(int m) {
    return fp16_for(m) ? 2 * (size_t)m + 32 : (size_t)m + 16;
}

// Workspace carve-up of one problem's arrays (its control block lives in the
// workspace header, see engine_header_bytes): returns bytes used from `base`.
__host__ inline size_t decode_ws_layout(int n, int m, ProblemDev *pd, char *base) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off = align_up(off + bytes, 256);
        return p;
    };
    char *touched = take((size_t)m);
    char *in_slots = take((size_t)n);
    char *slots = take((size_t)m * kSlotRec * 4);
    char *fp = take(fp_bytes(m));
    char *r_next = take((size_t)m * 8);
    char *hits = take(align_up((size_t)n, 4));
    if (pd) {
        pd->hits = reinterpret_cast<uint32_t *>(hits);
        pd->r_next = reinterpret_cast<double *>(r_next);
        pd->fp = reinterpret_cast<uint8_t *>(fp);
        pd->touched = reinterpret_cast<uint8_t *>(touched);
        pd->in_slots = reinterpret_cast<uint8_t *>(in_slots);
        pd->slots = reinterpret_cast<int32_t *>(slots);
    }
    return off;
}

// Workspace header shared by every decode call: launch-wide sync words and
// the P control blocks (contiguous, so one memset clears them and one copy
// reads every result back), then engine scratch.
struct alignas(64) EngineSync {
    unsigned arrive;  // monotonic grid-barrier counter
    int error;        // ErrorBits of the launch
    int pad[14];
};
static_assert(sizeof(EngineSync) == 64, "EngineSync layout");

// ---- binary64 bit helpers ------------------------------------------------

// Bits of v with -0.0 folded onto +0.0, so that bit equality is value
// equality for every finite double and 0 means "zero".
__device__ __forceinline__ unsigned long long value_bits(double v) {
    unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
    return (b << 1) == 0ull ? 0ull : b;
}

// Unsigned key with the numeric order of the (non-NaN) doubles.
__device__ __forceinline__ unsigned long long order_key(unsigned long long b) {
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int ld_volatile(const int *p) {
    return *reinterpret_cast<const volatile int *>(p);
}

// ---- host-side error reporting -------------------------------------------

void set_last_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);

#define CCS_CUDA_TRY(expr)                                        \
    do {                                                          \
        cudaError_t _e = (expr);                                  \
        if (_e != cudaSuccess) return ::ccs::cuda_fail(_e, #expr); \
    } while (0)

int check_sizes(int32_t n, int32_t m, int32_t d);

// launch counting / optional event timing (ccs_profile.cu)
void count_launches(int k);
bool profiling();
int prof_start(int kind, cudaStream_t s);
void prof_stop(int slot, cudaStream_t s);
void prof_collect();
void prof_add(int kind, double ms);
void prof_keep_stamps(const unsigned long long *st, int count, int sub_base);

// host-driven loop (ccs_decode.cu)
int decode_host_loop(const ProblemDev &P, const ccs_params &p, ccs_result *out, cudaStream_t s);

// persistent engine (ccs_engine.cu).  The workspace starts with
// engine_header_bytes(P) bytes: EngineSync, P DecodeCtrl, engine scratch.
size_t engine_header_bytes(int P);
// Whether the problem, launched alone with these params, keeps its
// fingerprints in shared memory (false also when no launch shape fits).
bool engine_fp_fits(const ProblemDev &pd, const ccs_params &prm);
// Record the launch shape ccs_autotune picked for launches on device `dev`
// whose largest d is dmax and whose problems all keep (fits) or do not all
// keep shared-memory fingerprints.
void tuned_schedule_set(int dev, int dmax, bool fits, int schedule);
void tuned_schedule_reset();
DecodeCtrl *header_ctrl(char *ws, int p);
int engine_run(ProblemDev *pds, int P, const ccs_params &prm, ccs_result *out, char *ws,
               cudaStream_t s, ccs_result *dev_out = nullptr);
// Resume mode (serving): the control blocks live with each problem
// (pds[p].ctrl) and persist between launches; problems flagged kPdFresh are
// initialised, the others continue from their saved state; at most
// iter_budget iterations run; out[p].status is -1 for problems still
// running.  `hdr` needs engine_resume_header_bytes(P) bytes.
size_t engine_resume_header_bytes(int P);
// Graph of `groups` launches run in turn; pds holds group g's sizes[g]
// descriptors after those of the groups before it.
int engine_capture(ProblemDev *pds, const int *sizes, int groups, const ccs_params &prm, char *ws,
                   ccs_result *dev_out, cudaGraphExec_t *exec);
// The expander's construction in two enqueued parts (ccs_setup.cu), for
// callers that batch the read-back of the largest row degree.
int expander_build_async(int32_t n, int32_t m, int32_t d, uint64_t seed, int32_t *csc_rows,
                         int64_t *csr_ptr, int32_t *csr_cols, void *ws, cudaStream_t s,
                         int **max_deg_dev);
int expander_sort_rows(int32_t m, int64_t *csr_ptr, int32_t *csr_cols, int host_max,
                       cudaStream_t s);

int engine_resume(ProblemDev *pds, int P, const ccs_params &prm, int iter_budget, ccs_result *out,
                  char *hdr, cudaStream_t s);
// A multi-group batch with merged tails (see ccs_engine.cu), run now or
// captured in a CUDA graph.
int engine_run_phased(ProblemDev *pds, const int *sizes, int groups, int count,
                      const ccs_params &prm, int group_iters, char *ctrl_hdr, char *rhdr,
                      cudaStream_t s, ccs_result *dev_out, ccs_result *host_out);
int engine_capture_phased(ProblemDev *pds, const int *sizes, int groups, int count,
                          const ccs_params &prm, int group_iters, char *ctrl_hdr, char *rhdr,
                          ccs_result *dev_out, cudaGraphExec_t *exec);
int check_params(const ccs_params *p, int d);

}  // namespace ccs

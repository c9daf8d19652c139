// ccs_engine.cu -- Parallel-l0 (Alg. 2) in one persistent cooperative launch.
//
// One launch runs every iteration of one or many independent problems.  The
// grid is one CTA per SM (co-resident by cooperative launch); the phases of an
// iteration are separated by grid barriers:
//
//   init      x_hat <- 0, r <- y, fingerprints of r, ||y||_0
//   score     every column of every running problem: exact score (Eq. (15)
//             or Alg. 8) and, if accepted, x_hat_j += omega_j (apply).
//   residual  every touched row: r_i = y_i - ordered sum of its nonzero
//             x_hat_j, new fingerprint, exact change of ||r||_0
//   stop      every CTA applies the stop rule to every problem from the same
//             counters, so all CTAs agree without another barrier
//
// Score phase, per CTA and problem segment (a contiguous range of 32-column
// tiles):
//   - the problem's 8-bit residual fingerprints (m bytes) and the segment's
//     CSC row indices stream into shared memory by TMA bulk copies
//     (cp.async.bulk, mbarrier completion); the CSC goes through a ring of
//     stages so the next chunks are in flight while warps work on this one;
//   - each warp tests its 32 columns against the fingerprint bound (a value's
//     count never exceeds its fingerprint's count), from shared memory only;
//   - the few columns that may reach alpha are queued, then scored exactly,
//     lane-parallel across the CTA: d binary64 gathers of r each.
// Problems whose fingerprints do not fit shared memory score every column
// exactly from the same stages.
//
// Every wait (grid barrier, mbarrier) is bounded by the watchdog: on time-out
// the CTA records kErrWatchdog, gives its in-flight copies a bounded time to
// land, and returns; the host reports CCS_ETIMEOUT.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <tuple>
#include <vector>

#include "ccs_device.cuh"

namespace ccs {

constexpr int kTile = 32;
constexpr int kMaxBlocks = 1024;
constexpr int kMaxProblems = 4096;  // per launch: their status and weight prefix live on chip
constexpr int kMaxStampIters = 1024;
constexpr int kMaxStages = 6;
constexpr int kOvfCap = 512;       // overflow rows listed per CTA and segment
constexpr int kQueueCap = 2048;     // most candidate columns queued per CTA and segment
constexpr int kMinQueue = 256;      // fewest (more go through the inline exact path)
constexpr int kFlagSkipArrive = 1;  // test hook: CTA 0 never arrives at barrier 1
constexpr int kFpChunk = 32768;     // bytes per fingerprint bulk copy
constexpr int kSubBase = 3 * kMaxStampIters + 2;  // CTA-0 score sub-phase stamps start here

struct Segment {
    int prob, lo, hi, pad;  // tiles [lo, hi) of problem `prob`
};

struct EngineArgs {
    ProblemDev single;          // used when probs == nullptr (one problem)
    const ProblemDev *probs;    // P descriptors in device memory
    int P;
    int alpha, mode, max_iter;
    int fp_cap;                 // bytes of the shared fingerprint buffer
    int stages;                 // CSC ring depth
    int stage_bytes;            // bytes per stage (one tile per warp)
    int queue_cap;              // candidate entries (column + its d rows)
    EngineSync *sync;
    unsigned long long *stamps; // globaltimer after each barrier (or null)
    long long watchdog_ns;
    int debug_flags;
    ccs_result *dev_out;        // per-problem results in device memory (or null)
    int resume;                 // control blocks persist; only kPdFresh problems initialise
    int iter_budget;            // iterations this launch may run
};

// ---- device helpers --------------------------------------------------------

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple
// of 16), completion counted in bytes on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// try_wait that may suspend the thread for up to `hint_ns` while the phase
// is incomplete (it returns as soon as the phase completes), so waiting
// warps do not spin through issue slots.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, uint32_t parity,
                                                    uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase.  On time-out marks the launch failed.
__device__ __forceinline__ bool mbar_wait(const EngineArgs &a, uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (!mbar_try_wait_sleep(bar, parity, 20000u)) {
        if (globaltimer() - t0 > (unsigned long long)a.watchdog_ns) {
            atomicOr(&a.sync->error, kErrWatchdog);
            return false;
        }
    }
    return true;
}

// Grid barrier number `index` (0-based).  Returns false if the wait ran past
// the watchdog (or another CTA already gave up).
__device__ bool grid_barrier(const EngineArgs &a, unsigned index, bool arrive = true) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (arrive) {
            __threadfence();
            atomicAdd(&a.sync->arrive, 1u);
        }
        const unsigned target = (index + 1u) * gridDim.x;
        const unsigned long long t0 = globaltimer();
        while (ld_acquire(&a.sync->arrive) < target) {
            if (*reinterpret_cast<volatile int *>(&a.sync->error) != 0 ||
                globaltimer() - t0 > (unsigned long long)a.watchdog_ns) {
                atomicOr(&a.sync->error, kErrWatchdog);
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
        if (ok && a.stamps && blockIdx.x == 0 && index < 3u * kMaxStampIters + 1u)
            a.stamps[index] = globaltimer();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ const ProblemDev &problem(const EngineArgs &a, int p) {
    return a.probs ? a.probs[p] : a.single;
}

// A CTA that leaves early (a wait ran out) marks every device-side result.
__device__ __forceinline__ void fail_out(const EngineArgs &a) {
    if (a.dev_out && threadIdx.x == 0)
        for (int p = 0; p < a.P; ++p) a.dev_out[problem(a, p).out_slot].error = CCS_ETIMEOUT;
}

// ---- work partition -----------------------------------------------------
//
// Every phase splits the tiles of the problems that are still running into
// gridDim.x contiguous shares of equal weight (part_weight below gives a
// tile's weight).
// Each CTA computes the same prefix of weights over the problems in shared
// memory and takes the tiles whose starting weight falls in its share, so
// the shares follow the running set from one iteration to the next.

enum PartKind { kPartScore = 0, kPartRows = 1, kPartInitCols = 2, kPartInitRows = 3 };

__device__ __forceinline__ long long part_tiles(const ProblemDev &P, int kind) {
    return (kind == kPartScore || kind == kPartInitCols) ? (P.n + kTile - 1) / kTile
                                                         : (P.m + kTile - 1) / kTile;
}

// Score tiles weigh d (their columns' row indices), four times more when the
// problem's fingerprints are not in shared memory (every column then gathers
// its d values of r); row tiles weigh 1.
__device__ __forceinline__ long long part_weight(const ProblemDev &P, int kind) {
    if (kind != kPartScore) return 1;
    return (P.flags & kPdUseFp) ? P.d : 4 * P.d;
}

// Does problem P take part in a partition of this kind?  Iteration phases:
// the running problems.  Init: every problem, or in resume mode the fresh
// ones only.
__device__ __forceinline__ bool part_on(const EngineArgs &a, const ProblemDev &P, int8_t status,
                                        int kind) {
    if (kind >= kPartInitCols) return !a.resume || (P.flags & kPdFresh);
    return status == kRunning;
}

// pref[0..P]: exclusive prefix of the problems' weights (0 for problems
// that are not running, except in the init kinds).  Block-wide.
template <int THREADS>
__device__ __noinline__ void build_partition(const EngineArgs &a, const int8_t *status, long long *pref,
                                int kind) {
    __shared__ long long s_warp[THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int per = (a.P + THREADS - 1) / THREADS;
    const int p0 = threadIdx.x * per;
    long long mine = 0;
    for (int q = 0; q < per; ++q) {
        const int p = p0 + q;
        if (p < a.P) {
            const ProblemDev &P = problem(a, p);
            if (part_on(a, P, status[p], kind)) mine += part_tiles(P, kind) * part_weight(P, kind);
        }
    }
    long long inc = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    __syncthreads();  // previous readers of pref / s_warp are done
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    long long before = 0;
    for (int w = 0; w < warp; ++w) before += s_warp[w];
    long long run = before + inc - mine;  // exclusive prefix of this thread's first element
    for (int q = 0; q < per; ++q) {
        const int p = p0 + q;
        if (p < a.P) {
            pref[p] = run;
            const ProblemDev &P = problem(a, p);
            if (part_on(a, P, status[p], kind)) run += part_tiles(P, kind) * part_weight(P, kind);
        }
    }
    if (threadIdx.x == THREADS - 1) pref[a.P] = run;
    __syncthreads();
}

// Visit this CTA's segments (problem, tiles [lo, hi)) of a partition.
template <typename F>
__device__ __forceinline__ void for_my_segments(const EngineArgs &a, const int8_t *status,
                                                const long long *pref, int kind, F &&fn) {
    const long long W = pref[a.P];
    if (W == 0) return;
    const long long B0 = W * blockIdx.x / gridDim.x, B1 = W * (blockIdx.x + 1) / gridDim.x;
    int lo = 0, hi = a.P;  // first p with pref[p + 1] > B0
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (pref[mid + 1] > B0) hi = mid;
        else lo = mid + 1;
    }
    for (int p = lo; p < a.P && pref[p] < B1; ++p) {
        const ProblemDev &P = problem(a, p);
        if (!part_on(a, P, status[p], kind)) continue;
        const long long w = part_weight(P, kind), tiles = part_tiles(P, kind);
        const long long t0 = B0 > pref[p] ? (B0 - pref[p] + w - 1) / w : 0;
        const long long t1 = min(tiles, (B1 - pref[p] + w - 1) / w);
        if (t1 > t0) fn(p, P, (int)t0, (int)t1);
    }
}

// Shared-memory state of the score phase.
struct ScoreSmem {
    uint8_t *fp;       // fingerprints of the current problem
    char *stage;       // a.stages * a.stage_bytes
    int32_t *queue;    // candidate columns
    uint64_t *full;    // per stage: its chunk has landed (TMA transaction count)
    uint64_t *empty;   // per stage: every consumer warp is done with it
    uint64_t *fp_bar;  // fingerprint copy
    int *qn;           // queue length
    unsigned long long *acc;  // accepted pairs of this CTA in the current segment
};

// Columns [col0, col1) of chunk `c` of a segment (tiles lo + c*W .. +W).
__device__ __forceinline__ void chunk_cols(const ProblemDev &P, int lo, int hi, int c, int per,
                                           long long &col0, long long &col1) {
    const int t0 = lo + c * per;
    const int t1 = min(hi, t0 + per);
    col0 = (long long)t0 * kTile;
    col1 = min((long long)P.n, (long long)t1 * kTile);
}

// Issue chunk `c` into ring slot `slot`: the largest 16-byte multiple of its
// row indices by TMA (the consumer reads any remaining < 4 ints, which only
// occur at a problem's last column, from global memory).
__device__ __forceinline__ void issue_chunk(const EngineArgs &a, const ProblemDev &P, int lo,
                                            int hi, int c, int per, ScoreSmem &S, int slot) {
    long long col0, col1;
    chunk_cols(P, lo, hi, c, per, col0, col1);
    const uint32_t tma = (uint32_t)((col1 - col0) * P.d * 4) & ~15u;
    uint64_t *bar = &S.full[slot];
    mbar_expect_tx(bar, tma);
    if (tma) bulk_g2s(S.stage + (size_t)slot * a.stage_bytes, P.csc_rows + col0 * P.d, tma, bar);
}

// Exact score and apply of one column inside the stream (problems without
// shared-memory fingerprints, or a full queue); the rows are read again from
// global memory, so the stream loop keeps no copy of them.
template <int DMAX, bool kPrefilter>
__device__ __forceinline__ bool score_inline(const EngineArgs &a, const ProblemDev &P, int j) {
    const int d = P.d;
    int32_t rows[DMAX];
#pragma unroll
    for (int t = 0; t < DMAX; ++t) rows[t] = (t < d) ? __ldg(P.csc_rows + (size_t)j * d + t) : 0;
    unsigned long long omega;
    const bool acc = exact_score<DMAX, kPrefilter>(rows, d, P.r, a.alpha, a.mode, &omega);
    if (acc) apply_pair<DMAX>(P, j, rows, d, omega);
    return acc;
}

// Queued candidates: exact score, lane-parallel over the CTA.  The r
// gathers, x_hat_j and the in-slots flag go out in one round trip.
template <int DMAX>
__device__ __forceinline__ void score_queue(const EngineArgs &a, const ProblemDev &P,
                                         const int32_t *queue, int qn,
                                         unsigned long long *acc_smem, bool ok) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int d = P.d;
    for (int b0 = warp * 32; b0 < qn; b0 += blockDim.x) {
        const int idx = b0 + lane;
        bool acc = false;
        if (ok && idx < qn) {
            const int32_t *e = queue + idx * (DMAX + 1);
            const int j = e[0];
            int32_t rows[DMAX];
            unsigned long long v[DMAX];
#pragma unroll
            for (int t = 0; t < DMAX; ++t) rows[t] = e[1 + t];
#pragma unroll
            for (int t = 0; t < DMAX; ++t) v[t] = (t < d) ? value_bits(__ldcg(P.r + rows[t])) : 0ull;
            const double xj = __ldcg(P.x_hat + j);
            const uint8_t ins = __ldcg(P.in_slots + j);
            unsigned long long omega;
            acc = exact_score_values<DMAX>(v, d, a.alpha, a.mode, &omega);
            if (acc) apply_pair_loaded<DMAX>(P, j, rows, d, omega, xj, ins);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, acc);
        if (lane == 0 && bal) atomicAdd(acc_smem, (unsigned long long)__popc(bal));
    }
}

// Score phase of one segment.  Warp 0 is the producer: its lane 0 streams
// the fingerprints and the CSC chunks by TMA, refilling a stage as soon as
// every consumer warp has released it.  Warps 1.. consume one 32-column tile
// of each chunk: the fingerprint bound from shared memory, candidates into
// the queue.  Then every warp scores the queued candidates exactly.
template <int DMAX, int THREADS>
__device__ __forceinline__ void score_segment(const EngineArgs &a, const ProblemDev &P,
                                              int seg_lo, int seg_hi, int g, ScoreSmem &S,
                                              unsigned &chunk_seq, unsigned &fp_seq, bool &ok) {
    const Segment sg{0, seg_lo, seg_hi, 0};
    const int warps = blockDim.x >> 5;
    constexpr int kTpw = (THREADS == 512) ? 2 : 1;  // tiles per consumer warp and chunk
    const int per = (warps - 1) * kTpw;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int d = P.d;
    const bool use_fp = (P.flags & kPdUseFp) != 0;
    const int tiles = sg.hi - sg.lo;
    const int nchunks = (tiles + per - 1) / per;
    unsigned long long *acc_slot = &P.ctrl->acc[g & 3];

    __syncthreads();  // previous users of the queue and fingerprints are done
    if (threadIdx.x == 0) {
        *S.qn = 0;
        *S.acc = 0;
    }
    __syncthreads();

    if (warp == 0) {
        if (lane == 0 && ok) {
            if (use_fp) {
                const uint32_t total = (uint32_t)align_up((size_t)P.m, 16);
                mbar_expect_tx(S.fp_bar, total);
                for (uint32_t off = 0; off < total; off += kFpChunk)
                    bulk_g2s(S.fp + off, P.fp + off, min((uint32_t)kFpChunk, total - off), S.fp_bar);
            }
            for (int c = 0; c < nchunks; ++c) {
                const unsigned seq = chunk_seq + c;
                const int slot = seq % a.stages;
                if (!mbar_wait(a, &S.empty[slot], ((seq / a.stages) & 1u) ^ 1u)) {
                    ok = false;
                    break;
                }
                issue_chunk(a, P, sg.lo, sg.hi, c, per, S, slot);
            }
        }
    } else {
        if (use_fp) ok = ok && mbar_wait(a, S.fp_bar, fp_seq & 1u);
        if (a.stamps && blockIdx.x == 0 && threadIdx.x == 32 && g < kMaxStampIters)
            a.stamps[kSubBase + 3 * g] = globaltimer();
        for (int c = 0; c < nchunks; ++c) {
            const unsigned seq = chunk_seq + c;
            const int slot = seq % a.stages;
            ok = ok && mbar_wait(a, &S.full[slot], (seq / a.stages) & 1u);
            const int32_t *stage =
                reinterpret_cast<const int32_t *>(S.stage + (size_t)slot * a.stage_bytes);
            long long col0, col1;
            chunk_cols(P, sg.lo, sg.hi, c, per, col0, col1);
            // ints of this chunk that came by TMA; only a problem's last chunk
            // can end with up to 3 ints that did not
            const long long e_tma = (((col1 - col0) * d * 4) & ~15ll) / 4;
            const bool tail = e_tma != (col1 - col0) * d;
#pragma unroll
            for (int u = 0; u < kTpw; ++u) {
            const int tile = sg.lo + c * per + u * (warps - 1) + (warp - 1);
            bool acc = false;
            if (ok && tile < sg.hi) {
                const int base = tile * kTile;
                const int cols = min(kTile, P.n - base);
                if (lane < cols) {
                    const int j = base + lane;
                    const long long e0 = (long long)(j - col0) * d;  // first int of column j
                    int32_t rows[DMAX];
                    if (!tail) {
#pragma unroll
                        for (int t = 0; t < DMAX; ++t) rows[t] = (t < d) ? stage[e0 + t] : 0;
                    } else {
#pragma unroll
                        for (int t = 0; t < DMAX; ++t)
                            rows[t] = (t < d) ? ((e0 + t < e_tma) ? stage[e0 + t]
                                                                  : __ldg(P.csc_rows + (size_t)j * d + t))
                                              : 0;
                    }
                    bool inline_exact = true;
                    if (use_fp) {
                        inline_exact = false;
                        if (may_accept<DMAX>(S.fp, rows, d, a.alpha, a.mode)) {
                            const int q = atomicAdd(S.qn, 1);
                            if (q < a.queue_cap) {  // scored after the stream
                                int32_t *e = S.queue + q * (DMAX + 1);
                                e[0] = j;
#pragma unroll
                                for (int t = 0; t < DMAX; ++t) e[1 + t] = rows[t];
                            } else {
                                inline_exact = true;
                            }
                        }
                    }
                    // the 1024-thread instance (64 registers) serves only
                    // problems with shared-memory fingerprints, whose
                    // columns reach this point after the fingerprint test
                    if (inline_exact) acc = score_inline<DMAX, THREADS != 1024>(a, P, j);
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, acc);
            if (lane == 0 && bal) atomicAdd(S.acc, (unsigned long long)__popc(bal));
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.empty[slot]);  // this warp is done with the stage
        }
    }
    chunk_seq += nchunks;
    if (use_fp) ++fp_seq;
    __syncthreads();  // stream done, queue complete
    if (a.stamps && blockIdx.x == 0 && threadIdx.x == 0 && g < kMaxStampIters)
        a.stamps[kSubBase + 3 * g + 1] = globaltimer();

    score_queue<DMAX>(a, P, S.queue, min(*S.qn, a.queue_cap), S.acc, ok);
    // one global atomic per CTA and segment (all warps' counts summed on chip)
    __syncthreads();
    if (threadIdx.x == 0) {
        if (*S.acc) atomicAdd(acc_slot, *S.acc);
        if (a.stamps && blockIdx.x == 0 && g < kMaxStampIters)
            a.stamps[kSubBase + 3 * g + 2] = globaltimer();
    }
}

// One row of the residual phase.  The touched flag, the row's slot record,
// y_i and the old r_i are independent loads issued together; only touched
// rows then gather their contributors' x_hat_j.
// One row tile of the residual phase.  Rows with more contributors than
// their slot record holds are appended to the CTA's overflow list (summed
// afterwards, one warp a row); when the list is full the warp sums them
// itself.
__device__ __noinline__ long long residual_tile(const ProblemDev &P, int tile, int lane,
                                                int *ovf, int *ovf_n, int ovf_cap) {
    const int i = tile * kTile + lane;
    long long delta = 0;
    bool touched = false, over = false;
    int js[kSlotRec];
    double yi = 0.0, ro = 0.0, s = 0.0;
    if (i < P.m) {
        touched = __ldcg(P.touched + i) != 0;
        load_record(P, i, js);
        yi = __ldg(P.y + i);
        ro = __ldcg(P.r + i);
        over = touched && js[0] > kSlots;
        if (touched && !over) s = row_sum_from_record(P, i, js);
    }
    bool later = false;
    if (over) {
        const int q = atomicAdd(ovf_n, 1);
        if (q < ovf_cap) {
            ovf[q] = i;
            later = true;
        }
    }
    const double so = overflow_row_sums(P, over && !later, i, lane);
    if (touched && !later) {
        if (over) s = so;
        P.touched[i] = 0;
        const double rn = __dsub_rn(yi, s);
        delta = (long long)(rn != 0.0) - (long long)(ro != 0.0);
        P.r[i] = rn;
        P.fp[i] = fingerprint(rn);
    }
    return warp_sum_ll(delta);
}

// A listed overflow row, by one warp; returns the row's change of ||r||_0.
__device__ __noinline__ long long residual_overflow_row(const ProblemDev &P, int i, int lane) {
    const double s = warp_ordered_row_sum(P.csr_ptr, P.csr_cols, P.x_hat, i, lane);
    long long delta = 0;
    if (lane == 0) {
        const double rn = __dsub_rn(__ldg(P.y + i), s);
        const double ro = __ldcg(P.r + i);
        delta = (long long)(rn != 0.0) - (long long)(ro != 0.0);
        P.touched[i] = 0;
        P.r[i] = rn;
        P.fp[i] = fingerprint(rn);
    }
    return delta;
}

template <int DMAX, int THREADS>
__global__ void __launch_bounds__(THREADS, 1) k_engine(const __grid_constant__ EngineArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int kWarps = THREADS / 32;
    __shared__ __align__(8) uint64_t s_bars[2 * kMaxStages + 1];
    __shared__ int s_qn;
    __shared__ unsigned long long s_acc;
    __shared__ long long s_sum;
    __shared__ int s_ovf_n;
    __shared__ int s_ovf[kOvfCap];  // rows whose sum needs the whole CSR row
    ScoreSmem S;
    S.fp = smem;
    S.stage = reinterpret_cast<char *>(smem + a.fp_cap);
    S.queue = reinterpret_cast<int32_t *>(S.stage + (size_t)a.stages * a.stage_bytes);
    int8_t *s_status = reinterpret_cast<int8_t *>(
        reinterpret_cast<char *>(S.queue) + ((a.queue_cap * (DMAX + 1) * 4 + 15) / 16) * 16);
    long long *s_pref = reinterpret_cast<long long *>(
        reinterpret_cast<char *>(s_status) + ((a.P + 15) / 16) * 16);  // a.P + 1 entries
    int *s_base = reinterpret_cast<int *>(s_pref + a.P + 1);          // a.P entries
    S.full = s_bars;
    S.empty = s_bars + kMaxStages;
    S.fp_bar = &s_bars[2 * kMaxStages];
    S.qn = &s_qn;
    S.acc = &s_acc;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned bar = 0, chunk_seq = 0, fp_seq = 0;
    bool ok = true;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kMaxStages; ++s) {
            mbar_init(&S.full[s], 1);            // the producer's expect_tx arrival
            mbar_init(&S.empty[s], kWarps - 1);  // one arrival per consumer warp
        }
        mbar_init(S.fp_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // resume mode: the accepted-count rings are per launch (the control
    // blocks themselves persist); they are first used after the init barrier
    if (a.resume && blockIdx.x == 0)
        for (int p = threadIdx.x; p < a.P; p += THREADS)
            for (int q = 0; q < 4; ++q) problem(a, p).ctrl->acc[q] = 0;
    __syncthreads();

    // ---- init: x_hat <- 0, r <- y (Alg. 2, first line) --------------------
    if (!a.probs) {
        // one problem: grid-stride over its columns and rows
        const ProblemDev &P = a.single;
        const long long gtid = blockIdx.x * (long long)THREADS + threadIdx.x;
        const long long gstride = (long long)gridDim.x * THREADS;
        for (long long j = gtid; j < P.n; j += gstride) {
            P.x_hat[j] = 0.0;
            P.in_slots[j] = 0;
        }
        if (threadIdx.x == 0) s_sum = 0;
        __syncthreads();
        long long nz = 0;
        for (long long i = gtid; i < P.m; i += gstride) {
            const double v = __ldg(P.y + i);
            P.r[i] = v;
            P.fp[i] = fingerprint(v);
            P.touched[i] = 0;
            P.slots[(size_t)i * kSlotRec] = 0;
            nz += (v != 0.0);
        }
        nz = warp_sum_ll(nz);
        if (lane == 0 && nz)
            atomicAdd(reinterpret_cast<unsigned long long *>(&s_sum), (unsigned long long)nz);
        __syncthreads();
        if (threadIdx.x == 0 && s_sum)
            atomicAdd(reinterpret_cast<unsigned long long *>(&P.ctrl->r0), (unsigned long long)s_sum);
    } else {
        build_partition<THREADS>(a, s_status, s_pref, kPartInitCols);
        for_my_segments(a, s_status, s_pref, kPartInitCols,
                        [&](int, const ProblemDev &P, int t0, int t1) {
                            for (int t = t0 + warp; t < t1; t += kWarps) {
                                const int j = t * kTile + lane;
                                if (j < P.n) {
                                    P.x_hat[j] = 0.0;
                                    P.in_slots[j] = 0;
                                }
                            }
                        });
        build_partition<THREADS>(a, s_status, s_pref, kPartInitRows);
        for_my_segments(a, s_status, s_pref, kPartInitRows,
                        [&](int, const ProblemDev &P, int t0, int t1) {
                            if (threadIdx.x == 0) s_sum = 0;
                            __syncthreads();
                            for (int t = t0 + warp; t < t1; t += kWarps) {
                                const int i = t * kTile + lane;
                                long long nz = 0;
                                if (i < P.m) {
                                    const double v = __ldg(P.y + i);
                                    P.r[i] = v;
                                    P.fp[i] = fingerprint(v);
                                    P.touched[i] = 0;
                                    P.slots[(size_t)i * kSlotRec] = 0;
                                    nz = (v != 0.0);
                                }
                                nz = warp_sum_ll(nz);
                                if (lane == 0 && nz)
                                    atomicAdd(reinterpret_cast<unsigned long long *>(&s_sum),
                                              (unsigned long long)nz);
                            }
                            __syncthreads();
                            if (threadIdx.x == 0 && s_sum)
                                atomicAdd(reinterpret_cast<unsigned long long *>(&P.ctrl->r0),
                                          (unsigned long long)s_sum);
                        });
    }
    if (!grid_barrier(a, bar++)) {
        fail_out(a);
        return;
    }
    for (int p = threadIdx.x; p < a.P; p += THREADS) {
        const ProblemDev &P = problem(a, p);
        if (a.resume && !(P.flags & kPdFresh)) {
            // continues from an earlier launch
            s_status[p] = (int8_t)__ldcg(&P.ctrl->status);
            s_base[p] = __ldcg(&P.ctrl->iteration);
            continue;
        }
        const long long r0 = __ldcg(&P.ctrl->r0);
        const int st = (r0 == 0) ? CCS_CONVERGED : (a.max_iter == 0 ? CCS_MAX_ITER : kRunning);
        s_status[p] = (int8_t)st;
        s_base[p] = 0;
        if (blockIdx.x == 0) {
            P.ctrl->status = st;
            P.ctrl->iteration = 0;
            P.ctrl->max_iter = a.max_iter;
            if (P.r0_hist) P.r0_hist[0] = r0;
        }
    }
    __syncthreads();

    for (int g = 0; g < a.iter_budget; ++g) {
        int any = 0;
        for (int p = threadIdx.x; p < a.P; p += THREADS) any |= (s_status[p] == kRunning);
        if (!__syncthreads_or(any)) break;
        if (blockIdx.x == 0)
            for (int p = threadIdx.x; p < a.P; p += THREADS) problem(a, p).ctrl->acc[(g + 2) & 3] = 0;

        // ---- score + apply ------------------------------------------------
        if (!a.probs) {
            const long long tiles = (a.single.n + kTile - 1) / kTile;
            const int t0 = (int)(tiles * blockIdx.x / gridDim.x);
            const int t1 = (int)(tiles * (blockIdx.x + 1) / gridDim.x);
            if (t1 > t0) score_segment<DMAX, THREADS>(a, a.single, t0, t1, g, S, chunk_seq, fp_seq, ok);
        } else {
            build_partition<THREADS>(a, s_status, s_pref, kPartScore);
            for_my_segments(a, s_status, s_pref, kPartScore,
                            [&](int, const ProblemDev &P, int t0, int t1) {
                                if (!__syncthreads_and(ok)) return;
                                score_segment<DMAX, THREADS>(a, P, t0, t1, g, S, chunk_seq, fp_seq, ok);
                            });
        }
        if (!__syncthreads_and(ok)) {
            // a TMA wait ran out: give copies still in flight time to land, then leave
            if (threadIdx.x == 0) {
                const unsigned long long t0 = globaltimer();
                while (globaltimer() - t0 < 2000000ull) __nanosleep(1000);
            }
            __syncthreads();
            fail_out(a);
            return;
        }
        const bool skip = (a.debug_flags & kFlagSkipArrive) && blockIdx.x == 0 && g == 0;
        if (!grid_barrier(a, bar++, !skip) || skip) {
            fail_out(a);
            return;
        }

        // ---- residual + ||r||_0 ---------------------------------------------
        auto residual_segment = [&](const ProblemDev &P, int t0, int t1) {
            if (threadIdx.x == 0) {
                s_sum = 0;
                s_ovf_n = 0;
            }
            __syncthreads();
            for (int t = t0 + warp; t < t1; t += kWarps) {
                const long long delta = residual_tile(P, t, lane, s_ovf, &s_ovf_n, kOvfCap);
                if (lane == 0 && delta)
                    atomicAdd(reinterpret_cast<unsigned long long *>(&s_sum), (unsigned long long)delta);
            }
            __syncthreads();
            const int novf = min(s_ovf_n, kOvfCap);
            for (int q = warp; q < novf; q += kWarps) {
                const long long delta = residual_overflow_row(P, s_ovf[q], lane);
                if (lane == 0 && delta)
                    atomicAdd(reinterpret_cast<unsigned long long *>(&s_sum), (unsigned long long)delta);
            }
            __syncthreads();  // one global atomic per CTA and segment
            if (threadIdx.x == 0 && s_sum)
                atomicAdd(reinterpret_cast<unsigned long long *>(&P.ctrl->r0), (unsigned long long)s_sum);
        };
        if (!a.probs) {
            const long long tiles = (a.single.m + kTile - 1) / kTile;
            residual_segment(a.single, (int)(tiles * blockIdx.x / gridDim.x),
                             (int)(tiles * (blockIdx.x + 1) / gridDim.x));
        } else {
            build_partition<THREADS>(a, s_status, s_pref, kPartRows);
            for_my_segments(a, s_status, s_pref, kPartRows,
                            [&](int, const ProblemDev &P, int t0, int t1) { residual_segment(P, t0, t1); });
        }
        if (!grid_barrier(a, bar++)) {
            fail_out(a);
            return;
        }

        // ---- stop rule ("while not converged", three ways to stop) ----------
        for (int p = threadIdx.x; p < a.P; p += THREADS) {
            if (s_status[p] != kRunning) continue;
            const ProblemDev &P = problem(a, p);
            int st;
            if (__ldcg(&P.ctrl->acc[g & 3]) == 0) {
                st = CCS_STALLED;
            } else {
                const long long r0 = __ldcg(&P.ctrl->r0);
                const int it = s_base[p] + g + 1;
                st = (r0 == 0) ? CCS_CONVERGED : (it >= a.max_iter ? CCS_MAX_ITER : kRunning);
                if (blockIdx.x == 0) {
                    P.ctrl->iteration = it;
                    if (P.r0_hist) P.r0_hist[it] = r0;
                }
            }
            s_status[p] = (int8_t)st;
            if (blockIdx.x == 0 && st != kRunning) P.ctrl->status = st;
        }
        __syncthreads();
    }
    // every problem has stopped: CTA 0 publishes the results on the device
    if (a.dev_out && blockIdx.x == 0) {
        for (int p = threadIdx.x; p < a.P; p += THREADS) {
            const ProblemDev &P = problem(a, p);
            ccs_result res;
            res.status = P.ctrl->status;
            res.iterations = P.ctrl->iteration;
            res.r0_final = __ldcg(&P.ctrl->r0);
            res.error = __ldcg(&a.sync->error) ? CCS_ETIMEOUT : CCS_OK;
            res.reserved = 0;
            a.dev_out[P.out_slot] = res;
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

// Schedules: (threads per CTA, tiles per consumer warp and chunk).
//   1: 1024 threads, 1 tile  (d <= 8: at most 64 registers a thread)
//   2:  512 threads, 2 tiles (any d: up to 128 registers a thread)
//   3:  768 threads, 1 tile  (d <= 8: up to 85 registers a thread)
static int schedule_for(int dmax, int requested) {
    if (requested == 2 || dmax > 8) return 2;
    if (requested == 3) return 3;
    return 1;  // measured fastest for d <= 8
}

typedef void (*engine_fn)(const EngineArgs);

#define CCS_ENGINE_CASES(T)                                                                   \
    case 1: return k_engine<1, T>;   case 2: return k_engine<2, T>;                           \
    case 3: return k_engine<3, T>;   case 4: return k_engine<4, T>;                           \
    case 5: return k_engine<5, T>;   case 6: return k_engine<6, T>;                           \
    case 7: return k_engine<7, T>;   case 8: return k_engine<8, T>;

static engine_fn engine_kernel(int dmax, int schedule) {
    if (schedule == 1) {
        switch (dmax) { CCS_ENGINE_CASES(1024) default: return nullptr; }
    }
    if (schedule == 3) {
        switch (dmax) { CCS_ENGINE_CASES(768) default: return nullptr; }
    }
    switch (dmax) {
        CCS_ENGINE_CASES(512)
        case 9: return k_engine<9, 512>;
        case 10: return k_engine<10, 512>;
        case 11: return k_engine<11, 512>;
        case 12: return k_engine<12, 512>;
        case 13: return k_engine<13, 512>;
        case 14: return k_engine<14, 512>;
        case 15: return k_engine<15, 512>;
        case 16: return k_engine<16, 512>;
        default: return nullptr;
    }
}
#undef CCS_ENGINE_CASES

static size_t stamps_bytes() {
    return align_up(sizeof(unsigned long long) * (kSubBase + 3 * kMaxStampIters), 256);
}

static size_t sync_bytes(int P) {
    return align_up(sizeof(EngineSync) + sizeof(DecodeCtrl) * (size_t)P, 256);
}

size_t engine_header_bytes(int P) {
    size_t b = sync_bytes(P) + stamps_bytes();
    if (P > 1) b += align_up(sizeof(ProblemDev) * (size_t)P, 256);
    return b;
}

DecodeCtrl *header_ctrl(char *ws, int p) {
    return reinterpret_cast<DecodeCtrl *>(ws + sizeof(EngineSync)) + p;
}

// Launch-setting caches: fixed tables (no heap allocation), filled on first
// use per device and kernel.
struct DeviceInfo {
    int sms = 0;
    int coop = 0;
    bool valid = false;
};

constexpr int kMaxDevices = 64;

static DeviceInfo device_info(int dev) {
    static std::mutex mu;
    static DeviceInfo cache[kMaxDevices];
    std::lock_guard<std::mutex> lk(mu);
    DeviceInfo di;
    if (dev >= 0 && dev < kMaxDevices && cache[dev].valid) return cache[dev];
    cudaDeviceGetAttribute(&di.sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&di.coop, cudaDevAttrCooperativeLaunch, dev);
    di.valid = true;
    if (dev >= 0 && dev < kMaxDevices) cache[dev] = di;
    return di;
}

// Largest dynamic shared memory a launch of `fn` may use on `dev`: the
// device's opt-in limit per CTA minus the kernel's static shared memory.
// The kernel's attribute is raised to it once, so every later launch of any
// size up to it is allowed.  Returns 0 on failure.
static size_t max_dynamic_smem(int dev, engine_fn fn) {
    struct Entry {
        int dev;
        engine_fn fn;
        size_t lim;
    };
    static std::mutex mu;
    static Entry cache[256];
    static int used = 0;
    std::lock_guard<std::mutex> lk(mu);
    for (int e = 0; e < used; ++e)
        if (cache[e].dev == dev && cache[e].fn == fn) return cache[e].lim;
    int optin = 0;
    cudaFuncAttributes fa;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, fn) != cudaSuccess)
        return 0;
    const size_t lim = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim) != cudaSuccess)
        return 0;
    if (used < 256) cache[used++] = Entry{dev, fn, lim};
    return lim;
}

// Resident CTAs per SM for (kernel, dynamic smem), cached.
static int blocks_per_sm(int dev, engine_fn fn, int threads, size_t smem) {
    struct Entry {
        int dev;
        engine_fn fn;
        size_t smem;
        int per_sm;
    };
    static std::mutex mu;
    static Entry cache[1024];
    static int used = 0;
    std::lock_guard<std::mutex> lk(mu);
    for (int e = 0; e < used; ++e)
        if (cache[e].dev == dev && cache[e].fn == fn && cache[e].smem == smem) return cache[e].per_sm;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess)
        return -1;
    if (used < 1024) cache[used++] = Entry{dev, fn, smem, per_sm};
    return per_sm;
}

// Launch the engine on P problems whose arrays are already carved out in
// `pds` (ctrl pointers into the header of `ws`).  Fills out[0..P).
// Launch shape of one engine launch: kernel instance, threads, shared
// memory plan, grid.  Marks each problem's kPdUseFp flag.
struct LaunchPlan {
    engine_fn fn;
    int threads, stages, queue_cap, G;
    size_t fp_cap, stage_bytes, smem;
};

static int plan_launch(ProblemDev *pds, int P, const ccs_params &prm, LaunchPlan &L) {
    int dmax = 1;
    bool aligned = true;
    for (int p = 0; p < P; ++p) {
        dmax = std::max(dmax, pds[p].d);
        aligned &= (reinterpret_cast<uintptr_t>(pds[p].csc_rows) & 15u) == 0;
    }
    if (!aligned) {
        set_last_error("csc_rows must be 16-byte aligned for the persistent engine");
        return CCS_EINVAL;
    }
    int sched = schedule_for(dmax, prm.schedule);
    for (int attempt = 0; attempt < 2; ++attempt) {
    engine_fn fn = engine_kernel(dmax, sched);
    const int threads = sched == 1 ? 1024 : (sched == 3 ? 768 : 512);
    const int tpw = sched == 2 ? 2 : 1;  // kTpw of the kernel instance
    const int warps = threads / 32;
    int dev = 0;
    CCS_CUDA_TRY(cudaGetDevice(&dev));
    const size_t smem_limit = max_dynamic_smem(dev, fn);
    if (smem_limit == 0) {
        set_last_error("could not size the engine's shared memory");
        return CCS_ECUDA;
    }
    const size_t stage_bytes = align_up((size_t)(warps - 1) * tpw * kTile * dmax * 4, 128);
    const size_t entry = (size_t)(dmax + 1) * 4;  // one queued candidate
    const size_t status_bytes = align_up((size_t)P, 16) + sizeof(long long) * (size_t)(P + 1) +
                                sizeof(int) * (size_t)P;
    if (P > kMaxProblems) {
        set_last_error("at most %d problems per launch (got %d)", kMaxProblems, P);
        return CCS_EINVAL;
    }
    const size_t fixed = status_bytes + 256 + kMinQueue * entry;
    if (fixed + 2 * stage_bytes > smem_limit) {
        set_last_error("too many problems in one launch (%d)", P);
        return CCS_EINVAL;
    }
    // fingerprints in shared memory when they leave room for >= 2 CSC stages
    const size_t fp_budget = smem_limit - fixed - 2 * stage_bytes;
    size_t fp_cap = 0;
    for (int p = 0; p < P; ++p) {
        ProblemDev &pd = pds[p];
        const size_t need = align_up((size_t)pd.m, 16);
        pd.flags = (pd.flags & ~kPdUseFp) | (need <= fp_budget ? kPdUseFp : 0);
        if (pd.flags & kPdUseFp) fp_cap = std::max(fp_cap, need);
    }
    fp_cap = align_up(fp_cap, 128);
    bool all_fp = true;
    for (int p = 0; p < P; ++p) all_fp &= (pds[p].flags & kPdUseFp) != 0;
    if (sched == 1 && !all_fp) {
        sched = 3;  // problems without fingerprints need the exact-path prefilter
        continue;
    }
    const int stages =
        (int)std::min<size_t>(kMaxStages, (smem_limit - fixed - fp_cap) / stage_bytes);
    const size_t left = smem_limit - fp_cap - (size_t)stages * stage_bytes - status_bytes - 256;
    const int queue_cap = (int)std::min<size_t>(kQueueCap, (left - 16) / entry);
    const size_t smem = fp_cap + (size_t)stages * stage_bytes +
                        align_up((size_t)queue_cap * entry, 16) + status_bytes;

    const DeviceInfo di = device_info(dev);
    if (!di.coop) {
        set_last_error("device does not support cooperative launches");
        return CCS_ECUDA;
    }
    const int per_sm = blocks_per_sm(dev, fn, threads, smem);
    if (per_sm < 1) {
        set_last_error("engine kernel does not fit on an SM (smem %zu)", smem);
        return CCS_ECUDA;
    }
    const int G = std::min(kMaxBlocks, di.sms);
    L.fn = fn;
    L.threads = threads;
    L.stages = stages;
    L.queue_cap = queue_cap;
    L.G = G;
    L.fp_cap = fp_cap;
    L.stage_bytes = stage_bytes;
    L.smem = smem;
    return CCS_OK;
    }
    set_last_error("no launch shape fits");
    return CCS_EINVAL;
}

static void fill_args(EngineArgs &a, const LaunchPlan &L, int P, const ccs_params &prm) {
    std::memset(&a, 0, sizeof(a));
    a.P = P;
    a.alpha = prm.alpha;
    a.mode = prm.score_mode;
    a.max_iter = prm.max_iter;
    a.fp_cap = (int)L.fp_cap;
    a.stages = L.stages;
    a.stage_bytes = (int)L.stage_bytes;
    a.queue_cap = L.queue_cap;
    a.watchdog_ns = (long long)(prm.watchdog_ms > 0 ? prm.watchdog_ms : 2000) * 1000000ll;
    a.debug_flags = prm.debug_flags;
    a.iter_budget = 0x7fffffff;
}


int engine_run(ProblemDev *pds, int P, const ccs_params &prm, ccs_result *out, char *ws,
               cudaStream_t s, ccs_result *dev_out) {
    LaunchPlan L;
    int rc = plan_launch(pds, P, prm, L);
    if (rc) return rc;
    EngineArgs a;
    fill_args(a, L, P, prm);
    a.sync = reinterpret_cast<EngineSync *>(ws);
    char *e = ws + sync_bytes(P);
    unsigned long long *stamps = reinterpret_cast<unsigned long long *>(e);
    e += stamps_bytes();
    a.stamps = (profiling() && !dev_out) ? stamps : nullptr;
    a.dev_out = dev_out;
    if (a.stamps) CCS_CUDA_TRY(cudaMemsetAsync(stamps, 0, stamps_bytes(), s));

    // barrier state and control blocks start at zero
    CCS_CUDA_TRY(cudaMemsetAsync(ws, 0, sync_bytes(P), s));

    if (P == 1) {
        a.single = pds[0];
        a.probs = nullptr;
    } else {
        ProblemDev *d_probs = reinterpret_cast<ProblemDev *>(e);
        e += align_up(sizeof(ProblemDev) * (size_t)P, 256);
        CCS_CUDA_TRY(cudaMemcpyAsync(d_probs, pds, sizeof(ProblemDev) * P,
                                     cudaMemcpyHostToDevice, s));
        a.probs = d_probs;
    }

    void *args[] = {&a};
    const int ev = prof_start(CCS_K_PERSISTENT, s);
    CCS_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)L.fn, dim3(L.G), dim3(L.threads), args,
                                             L.smem, s));
    prof_stop(ev, s);
    count_launches(1);
    if (dev_out) return CCS_OK;  // asynchronous: the kernel writes the results

    // results: one copy of the sync word and every control block (a stack
    // buffer for small launches, so single decodes allocate nothing)
    const size_t hdr_bytes = sizeof(EngineSync) + sizeof(DecodeCtrl) * (size_t)P;
    alignas(64) char hdr_small[sizeof(EngineSync) + sizeof(DecodeCtrl) * 8];
    std::vector<char> hdr_big;
    char *hdr = hdr_small;
    if (P > 8) {
        hdr_big.resize(hdr_bytes);
        hdr = hdr_big.data();
    }
    CCS_CUDA_TRY(cudaMemcpyAsync(hdr, ws, hdr_bytes, cudaMemcpyDeviceToHost, s));
    std::vector<unsigned long long> hst;
    if (a.stamps) {
        hst.resize(kSubBase + 3 * kMaxStampIters);
        CCS_CUDA_TRY(cudaMemcpyAsync(hst.data(), stamps, sizeof(unsigned long long) * hst.size(),
                                     cudaMemcpyDeviceToHost, s));
    }
    CCS_CUDA_TRY(cudaStreamSynchronize(s));
    EngineSync hs;
    std::memcpy(&hs, hdr, sizeof(hs));
    const int herr = hs.error;
    int max_it = 0;
    for (int p = 0; p < P; ++p) {
        DecodeCtrl hc;
        std::memcpy(&hc, hdr + sizeof(EngineSync) + sizeof(DecodeCtrl) * (size_t)p, sizeof(hc));
        out[p].status = hc.status;
        out[p].iterations = hc.iteration;
        out[p].r0_final = hc.r0;
        out[p].error = herr ? CCS_ETIMEOUT : CCS_OK;
        out[p].reserved = 0;
        max_it = std::max(max_it, hc.iteration);
    }
    if (a.stamps) prof_keep_stamps(hst.data(), (int)hst.size(), kSubBase);
    if (a.stamps && !herr) {
        // barrier 0 ends init; iteration g: score ends at 1+2g, residual at 2+2g
        for (int g = 0; g < max_it && 2 + 2 * g < (int)hst.size(); ++g) {
            const unsigned long long t0 = hst[2 * g], t1 = hst[1 + 2 * g], t2 = hst[2 + 2 * g];
            if (t1 >= t0 && t2 >= t1 && t0) {
                prof_add(CCS_K_SCORE, (t1 - t0) * 1e-6);
                prof_add(CCS_K_RESIDUAL, (t2 - t1) * 1e-6);
                // CTA 0's view of the score phase: fingerprints in, stream
                // done, queue done (0 when it had nothing to score)
                const unsigned long long f = hst[kSubBase + 3 * g], st = hst[kSubBase + 3 * g + 1],
                                         q = hst[kSubBase + 3 * g + 2];
                if (f >= t0 && st >= f && q >= st && q <= t1) {
                    prof_add(CCS_K_PHASE_FP, (f - t0) * 1e-6);
                    prof_add(CCS_K_PHASE_STREAM, (st - f) * 1e-6);
                    prof_add(CCS_K_PHASE_QUEUE, (q - st) * 1e-6);
                }
            }
        }
    }
    if (herr) {
        set_last_error("a bounded device wait exceeded the watchdog (%d ms)",
                       prm.watchdog_ms > 0 ? prm.watchdog_ms : 2000);
        return CCS_ETIMEOUT;
    }
    return CCS_OK;
}

// Capture decode launches (header memset + cooperative kernel, one pair per
// group, run one after the other) into a CUDA graph.  pds holds the groups'
// descriptors back to back, group g's sizes[g] of them, each with its control
// block at the group's own index in the header.  The descriptors are uploaded
// now, outside the capture, to disjoint places of the header; the graph bakes
// the workspace and array pointers.  Results go to dev_out.
int engine_capture(ProblemDev *pds, const int *sizes, int groups, const ccs_params &prm, char *ws,
                   ccs_result *dev_out, cudaGraphExec_t *exec) {
    int total = 0;
    for (int g = 0; g < groups; ++g) total += sizes[g];
    std::vector<EngineArgs> args(groups);
    std::vector<LaunchPlan> plans(groups);
    ProblemDev *d_probs = reinterpret_cast<ProblemDev *>(ws + sync_bytes(total) + stamps_bytes());
    for (int g = 0, first = 0; g < groups; first += sizes[g], ++g) {
        const int P = sizes[g];
        int rc = plan_launch(pds + first, P, prm, plans[g]);
        if (rc) return rc;
        EngineArgs &a = args[g];
        fill_args(a, plans[g], P, prm);
        a.sync = reinterpret_cast<EngineSync *>(ws);
        a.dev_out = dev_out;
        a.stamps = nullptr;
        if (P == 1) {
            a.single = pds[first];
            a.probs = nullptr;
        } else {
            a.probs = d_probs + first;
        }
    }
    // upload the descriptors with the flags plan_launch set
    if (total > 1)
        CCS_CUDA_TRY(cudaMemcpy(d_probs, pds, sizeof(ProblemDev) * total, cudaMemcpyHostToDevice));
    cudaStream_t cs;
    CCS_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e1 = cudaSuccess;
        for (int g = 0; g < groups && e1 == cudaSuccess; ++g) {
            const LaunchPlan &L = plans[g];
            void *kargs[] = {&args[g]};
            e1 = cudaMemsetAsync(ws, 0, sync_bytes(sizes[g]), cs);
            if (e1 == cudaSuccess)
                e1 = cudaLaunchCooperativeKernel((const void *)L.fn, dim3(L.G), dim3(L.threads),
                                                 kargs, L.smem, cs);
        }
        e = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = e1;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return cuda_fail(e, "capturing the engine launch");
    return CCS_OK;
}

// Resume-mode header: [EngineSync | P ccs_result] [stamps] [P descriptors].
static size_t resume_results_bytes(int P) {
    return align_up(sizeof(EngineSync) + sizeof(ccs_result) * (size_t)P, 256);
}

size_t engine_resume_header_bytes(int P) {
    return resume_results_bytes(P) + stamps_bytes() + align_up(sizeof(ProblemDev) * (size_t)P, 256);
}

int engine_resume(ProblemDev *pds, int P, const ccs_params &prm, int iter_budget, ccs_result *out,
                  char *hdr, cudaStream_t s) {
    LaunchPlan L;
    int rc = plan_launch(pds, P, prm, L);
    if (rc) return rc;
    EngineArgs a;
    fill_args(a, L, P, prm);
    a.resume = 1;
    a.iter_budget = iter_budget > 0 ? iter_budget : 1;
    a.sync = reinterpret_cast<EngineSync *>(hdr);
    a.dev_out = reinterpret_cast<ccs_result *>(hdr + sizeof(EngineSync));
    ProblemDev *d_probs =
        reinterpret_cast<ProblemDev *>(hdr + resume_results_bytes(P) + stamps_bytes());
    a.probs = d_probs;
    CCS_CUDA_TRY(cudaMemsetAsync(hdr, 0, sizeof(EngineSync), s));
    CCS_CUDA_TRY(cudaMemcpyAsync(d_probs, pds, sizeof(ProblemDev) * P, cudaMemcpyHostToDevice, s));
    void *args[] = {&a};
    const int ev = prof_start(CCS_K_PERSISTENT, s);
    CCS_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)L.fn, dim3(L.G), dim3(L.threads), args,
                                             L.smem, s));
    prof_stop(ev, s);
    count_launches(1);
    const size_t bytes = sizeof(EngineSync) + sizeof(ccs_result) * (size_t)P;
    std::vector<char> h(bytes);
    CCS_CUDA_TRY(cudaMemcpyAsync(h.data(), hdr, bytes, cudaMemcpyDeviceToHost, s));
    CCS_CUDA_TRY(cudaStreamSynchronize(s));
    EngineSync hs;
    std::memcpy(&hs, h.data(), sizeof(hs));
    std::memcpy(out, h.data() + sizeof(EngineSync), sizeof(ccs_result) * (size_t)P);
    if (hs.error) {
        for (int p = 0; p < P; ++p) out[p].error = CCS_ETIMEOUT;
        set_last_error("a bounded device wait exceeded the watchdog");
        return CCS_ETIMEOUT;
    }
    return CCS_OK;
}

}  // namespace ccs

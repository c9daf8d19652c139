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
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "ccs_device.cuh"

namespace ccs {

constexpr int kTile = 32;
constexpr int kMaxBlocks = 1024;
constexpr int kMaxStampIters = 1024;
constexpr int kMaxStages = 6;
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
    const int *score_ptr;       // G+1 offsets into score_segs (batch only)
    const Segment *score_segs;
    const int *res_ptr;
    const Segment *res_segs;
    EngineSync *sync;
    unsigned long long *stamps; // globaltimer after each barrier (or null)
    long long watchdog_ns;
    int debug_flags;
    ccs_result *dev_out;        // per-problem results in device memory (or null)
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

// Bounded wait on an mbarrier phase.  On time-out marks the launch failed.
__device__ __forceinline__ bool mbar_wait(const EngineArgs &a, uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (!mbar_try_wait(bar, parity)) {
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
        for (int p = 0; p < a.P; ++p) a.dev_out[p].error = CCS_ETIMEOUT;
}

// This CTA's segments of a phase.  One problem: a contiguous share of its
// tiles computed here; a batch: the host-built partition.
struct SegList {
    const Segment *segs;
    int count;
    Segment one;
};

__device__ __forceinline__ SegList my_segments(const EngineArgs &a, bool score) {
    SegList L;
    if (!a.probs) {
        const ProblemDev &P = a.single;
        const long long tiles = score ? (P.n + kTile - 1) / kTile : (P.m + kTile - 1) / kTile;
        L.one.prob = 0;
        L.one.lo = (int)(tiles * blockIdx.x / gridDim.x);
        L.one.hi = (int)(tiles * (blockIdx.x + 1) / gridDim.x);
        L.one.pad = 0;
        L.segs = nullptr;
        L.count = 1;
    } else {
        const int *ptr = score ? a.score_ptr : a.res_ptr;
        L.segs = (score ? a.score_segs : a.res_segs) + ptr[blockIdx.x];
        L.count = ptr[blockIdx.x + 1] - ptr[blockIdx.x];
        L.one = Segment{0, 0, 0, 0};
    }
    return L;
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

// Score phase of one segment.  Warp 0 is the producer: its lane 0 streams
// the fingerprints and the CSC chunks by TMA, refilling a stage as soon as
// every consumer warp has released it.  Warps 1.. consume one 32-column tile
// of each chunk: the fingerprint bound from shared memory, candidates into
// the queue.  Then every warp scores the queued candidates exactly.
template <int DMAX>
__device__ __forceinline__ void score_segment(const EngineArgs &a, const ProblemDev &P,
                                              const Segment &sg, int g, ScoreSmem &S,
                                              unsigned &chunk_seq, unsigned &fp_seq, bool &ok) {
    const int warps = blockDim.x >> 5;
    const int per = warps - 1;  // tiles per chunk: one per consumer warp
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int d = P.d;
    const bool use_fp = P.pad != 0;
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
            const long long e_tma = (((col1 - col0) * d * 4) & ~15ll) / 4;  // ints that came by TMA
            const int tile = sg.lo + c * per + (warp - 1);
            bool acc = false;
            if (ok && tile < sg.hi) {
                const int base = tile * kTile;
                const int cols = min(kTile, P.n - base);
                if (lane < cols) {
                    const int j = base + lane;
                    const long long e0 = (long long)(j - col0) * d;  // first int of column j
                    int32_t rows[DMAX];
#pragma unroll
                    for (int t = 0; t < DMAX; ++t)
                        rows[t] = (t < d) ? ((e0 + t < e_tma) ? stage[e0 + t]
                                                              : __ldg(P.csc_rows + (size_t)j * d + t))
                                          : 0;
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
                    if (inline_exact) {
                        unsigned long long omega;
                        acc = exact_score<DMAX>(rows, d, P.r, a.alpha, a.mode, &omega);
                        if (acc) apply_pair<DMAX>(P, j, rows, d, omega);
                    }
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, acc);
            if (lane == 0 && bal) atomicAdd(S.acc, (unsigned long long)__popc(bal));
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.empty[slot]);  // this warp is done with the stage
        }
    }
    chunk_seq += nchunks;
    if (use_fp) ++fp_seq;
    __syncthreads();  // stream done, queue complete
    if (a.stamps && blockIdx.x == 0 && threadIdx.x == 0 && g < kMaxStampIters)
        a.stamps[kSubBase + 3 * g + 1] = globaltimer();

    // queued candidates: exact score, lane-parallel over the CTA.  The r
    // gathers, x_hat_j and the in-slots flag go out in one round trip.
    const int qn = min(*S.qn, a.queue_cap);
    for (int b0 = warp * 32; b0 < qn; b0 += blockDim.x) {
        const int idx = b0 + lane;
        bool acc = false;
        if (ok && idx < qn) {
            const int32_t *e = S.queue + idx * (DMAX + 1);
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
        if (lane == 0 && bal) atomicAdd(S.acc, (unsigned long long)__popc(bal));
    }
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
__device__ __forceinline__ long long residual_tile(const ProblemDev &P, int tile, int lane) {
    const int i = tile * kTile + lane;
    long long delta = 0;
    if (i < P.m) {
        const uint8_t touched = __ldcg(P.touched + i);
        int js[kSlotRec];
        load_record(P, i, js);
        const double yi = __ldg(P.y + i);
        const double ro = __ldcg(P.r + i);
        if (touched) {
            P.touched[i] = 0;
            const double rn = __dsub_rn(yi, row_sum_from_record(P, i, js));
            delta = (long long)(rn != 0.0) - (long long)(ro != 0.0);
            P.r[i] = rn;
            P.fp[i] = fingerprint(rn);
        }
    }
    return warp_sum_ll(delta);
}

template <int DMAX, int THREADS>
__global__ void __launch_bounds__(THREADS, 1) k_engine(const __grid_constant__ EngineArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int kWarps = THREADS / 32;
    __shared__ __align__(8) uint64_t s_bars[2 * kMaxStages + 1];
    __shared__ int s_qn;
    __shared__ unsigned long long s_acc;
    __shared__ long long s_sum;
    ScoreSmem S;
    S.fp = smem;
    S.stage = reinterpret_cast<char *>(smem + a.fp_cap);
    S.queue = reinterpret_cast<int32_t *>(S.stage + (size_t)a.stages * a.stage_bytes);
    int8_t *s_status = reinterpret_cast<int8_t *>(S.queue + a.queue_cap * (DMAX + 1));
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
    __syncthreads();

    // ---- init: x_hat <- 0, r <- y (Alg. 2, first line) --------------------
    const long long gtid = blockIdx.x * (long long)THREADS + threadIdx.x;
    const long long gstride = (long long)gridDim.x * THREADS;
    for (int p = 0; p < a.P; ++p) {
        const ProblemDev &P = problem(a, p);
        if (threadIdx.x == 0) s_sum = 0;
        __syncthreads();
        for (long long j = gtid; j < P.n; j += gstride) {
            P.x_hat[j] = 0.0;
            P.in_slots[j] = 0;
        }
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
        if (lane == 0 && nz) atomicAdd(reinterpret_cast<unsigned long long *>(&s_sum), (unsigned long long)nz);
        __syncthreads();
        if (threadIdx.x == 0 && s_sum)
            atomicAdd(reinterpret_cast<unsigned long long *>(&P.ctrl->r0), (unsigned long long)s_sum);
    }
    if (!grid_barrier(a, bar++)) {
        fail_out(a);
        return;
    }
    for (int p = threadIdx.x; p < a.P; p += THREADS) {
        const ProblemDev &P = problem(a, p);
        const long long r0 = __ldcg(&P.ctrl->r0);
        const int st = (r0 == 0) ? CCS_CONVERGED : (a.max_iter == 0 ? CCS_MAX_ITER : kRunning);
        s_status[p] = (int8_t)st;
        if (blockIdx.x == 0) {
            P.ctrl->status = st;
            P.ctrl->iteration = 0;
            P.ctrl->max_iter = a.max_iter;
            if (P.r0_hist) P.r0_hist[0] = r0;
        }
    }
    __syncthreads();

    for (int g = 0;; ++g) {
        int any = 0;
        for (int p = threadIdx.x; p < a.P; p += THREADS) any |= (s_status[p] == kRunning);
        if (!__syncthreads_or(any)) break;
        if (blockIdx.x == 0)
            for (int p = threadIdx.x; p < a.P; p += THREADS) problem(a, p).ctrl->acc[(g + 2) & 3] = 0;

        // ---- score + apply ------------------------------------------------
        {
            const SegList L = my_segments(a, true);
            for (int s = 0; s < L.count; ++s) {
                const Segment sg = L.segs ? L.segs[s] : L.one;
                if (s_status[sg.prob] != kRunning || sg.hi <= sg.lo) continue;
                score_segment<DMAX>(a, problem(a, sg.prob), sg, g, S, chunk_seq, fp_seq, ok);
                if (!__syncthreads_and(ok)) break;
            }
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
        {
            const SegList L = my_segments(a, false);
            for (int s = 0; s < L.count; ++s) {
                const Segment sg = L.segs ? L.segs[s] : L.one;
                if (s_status[sg.prob] != kRunning) continue;
                const ProblemDev &P = problem(a, sg.prob);
                if (threadIdx.x == 0) s_sum = 0;
                __syncthreads();
                for (int t = sg.lo + warp; t < sg.hi; t += kWarps) {
                    const long long delta = residual_tile(P, t, lane);
                    if (lane == 0 && delta)
                        atomicAdd(reinterpret_cast<unsigned long long *>(&s_sum), (unsigned long long)delta);
                }
                __syncthreads();  // one global atomic per CTA and segment
                if (threadIdx.x == 0 && s_sum)
                    atomicAdd(reinterpret_cast<unsigned long long *>(&P.ctrl->r0),
                              (unsigned long long)s_sum);
            }
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
                const int it = g + 1;
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
            a.dev_out[p] = res;
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

static int threads_for(int dmax) { return dmax <= 8 ? 1024 : 512; }

typedef void (*engine_fn)(const EngineArgs);

static engine_fn engine_kernel(int dmax) {
    switch (dmax) {
        case 1: return k_engine<1, 1024>;
        case 2: return k_engine<2, 1024>;
        case 3: return k_engine<3, 1024>;
        case 4: return k_engine<4, 1024>;
        case 5: return k_engine<5, 1024>;
        case 6: return k_engine<6, 1024>;
        case 7: return k_engine<7, 1024>;
        case 8: return k_engine<8, 1024>;
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

static size_t stamps_bytes() {
    return align_up(sizeof(unsigned long long) * (kSubBase + 3 * kMaxStampIters), 256);
}

static size_t sync_bytes(int P) {
    return align_up(sizeof(EngineSync) + sizeof(DecodeCtrl) * (size_t)P, 256);
}

size_t engine_header_bytes(int P) {
    size_t b = sync_bytes(P) + stamps_bytes();
    if (P > 1) {
        b += align_up(sizeof(ProblemDev) * (size_t)P, 256);
        b += 2 * align_up(sizeof(int) * (kMaxBlocks + 1), 256);
        b += 2 * align_up(sizeof(Segment) * (size_t)(kMaxBlocks + P), 256);
    }
    return b;
}

DecodeCtrl *header_ctrl(char *ws, int p) {
    return reinterpret_cast<DecodeCtrl *>(ws + sizeof(EngineSync)) + p;
}

struct DeviceInfo {
    int sms = 0;
    int coop = 0;
};

static DeviceInfo device_info(int dev) {
    static std::mutex mu;
    static std::map<int, DeviceInfo> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    DeviceInfo di;
    cudaDeviceGetAttribute(&di.sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&di.coop, cudaDevAttrCooperativeLaunch, dev);
    cache[dev] = di;
    return di;
}

// Largest dynamic shared memory a launch of `fn` may use on `dev`: the
// device's opt-in limit per CTA minus the kernel's static shared memory.
// The kernel's attribute is raised to it once, so every later launch of any
// size up to it is allowed.  Returns 0 on failure.
static size_t max_dynamic_smem(int dev, engine_fn fn) {
    static std::mutex mu;
    static std::map<std::pair<int, void *>, size_t> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(dev, (void *)fn);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int optin = 0;
    cudaFuncAttributes fa;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, fn) != cudaSuccess)
        return 0;
    const size_t lim = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim) != cudaSuccess)
        return 0;
    cache[key] = lim;
    return lim;
}

// Resident CTAs per SM for (kernel, dynamic smem), cached.
static int blocks_per_sm(int dev, engine_fn fn, int threads, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<int, void *, size_t>, int> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_tuple(dev, (void *)fn, smem);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess)
        return -1;
    cache[key] = per_sm;
    return per_sm;
}

// Split P problems' tiles (weight w_p each) into G contiguous shares.
static void partition(const std::vector<long long> &tiles, const std::vector<int> &weight, int G,
                      std::vector<int> &ptr, std::vector<Segment> &segs) {
    std::vector<std::vector<Segment>> per(G);
    long long W = 0;
    for (size_t p = 0; p < tiles.size(); ++p) W += tiles[p] * weight[p];
    long long S = 0;  // weight before problem p
    for (size_t p = 0; p < tiles.size(); ++p) {
        const long long c = tiles[p], w = weight[p];
        if (c == 0) continue;
        auto first_tile = [&](long long b) -> long long {  // first tile with start*G >= b*W
            long long num = b * W - S * G;
            if (num <= 0) return 0;
            long long t = (num + w * G - 1) / (w * G);
            return std::min(t, c);
        };
        long long b0 = std::min<long long>(G - 1, (S * G) / std::max<long long>(W, 1));
        long long b1 = std::min<long long>(G - 1, ((S + (c - 1) * w) * G) / std::max<long long>(W, 1));
        for (long long b = b0; b <= b1; ++b) {
            const long long lo = first_tile(b), hi = (b == G - 1) ? c : first_tile(b + 1);
            if (hi > lo) per[b].push_back(Segment{(int)p, (int)lo, (int)hi, 0});
        }
        S += c * w;
    }
    ptr.assign(G + 1, 0);
    segs.clear();
    for (int b = 0; b < G; ++b) {
        ptr[b] = (int)segs.size();
        segs.insert(segs.end(), per[b].begin(), per[b].end());
    }
    ptr[G] = (int)segs.size();
}

// Launch the engine on P problems whose arrays are already carved out in
// `pds` (ctrl pointers into the header of `ws`).  Fills out[0..P).
int engine_run(std::vector<ProblemDev> &pds, const ccs_params &prm, ccs_result *out, char *ws,
               cudaStream_t s, ccs_result *dev_out) {
    const int P = (int)pds.size();
    int dmax = 1;
    bool aligned = true;
    for (auto &pd : pds) {
        dmax = std::max(dmax, pd.d);
        aligned &= (reinterpret_cast<uintptr_t>(pd.csc_rows) & 15u) == 0;
    }
    if (!aligned) {
        set_last_error("csc_rows must be 16-byte aligned for the persistent engine");
        return CCS_EINVAL;
    }
    engine_fn fn = engine_kernel(dmax);
    const int threads = threads_for(dmax);
    const int warps = threads / 32;
    int dev = 0;
    CCS_CUDA_TRY(cudaGetDevice(&dev));
    const size_t smem_limit = max_dynamic_smem(dev, fn);
    if (smem_limit == 0) {
        set_last_error("could not size the engine's shared memory");
        return CCS_ECUDA;
    }
    const size_t stage_bytes = align_up((size_t)(warps - 1) * kTile * dmax * 4, 128);
    const size_t entry = (size_t)(dmax + 1) * 4;  // one queued candidate
    const size_t status_bytes = align_up((size_t)P, 16);
    const size_t fixed = status_bytes + 256 + kMinQueue * entry;
    if (fixed + 2 * stage_bytes > smem_limit) {
        set_last_error("too many problems in one launch (%d)", P);
        return CCS_EINVAL;
    }
    // fingerprints in shared memory when they leave room for >= 2 CSC stages
    const size_t fp_budget = smem_limit - fixed - 2 * stage_bytes;
    size_t fp_cap = 0;
    for (auto &pd : pds) {
        const size_t need = align_up((size_t)pd.m, 16);
        pd.pad = need <= fp_budget ? 1 : 0;
        if (pd.pad) fp_cap = std::max(fp_cap, need);
    }
    fp_cap = align_up(fp_cap, 128);
    const int stages =
        (int)std::min<size_t>(kMaxStages, (smem_limit - fixed - fp_cap) / stage_bytes);
    const size_t left = smem_limit - fp_cap - (size_t)stages * stage_bytes - status_bytes - 256;
    const int queue_cap = (int)std::min<size_t>(kQueueCap, left / entry);
    const size_t smem = fp_cap + (size_t)stages * stage_bytes + (size_t)queue_cap * entry +
                        status_bytes;

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

    EngineArgs a;
    std::memset(&a, 0, sizeof(a));
    a.P = P;
    a.alpha = prm.alpha;
    a.mode = prm.score_mode;
    a.max_iter = prm.max_iter;
    a.fp_cap = (int)fp_cap;
    a.stages = stages;
    a.stage_bytes = (int)stage_bytes;
    a.queue_cap = queue_cap;
    a.watchdog_ns = (long long)(prm.watchdog_ms > 0 ? prm.watchdog_ms : 2000) * 1000000ll;
    a.debug_flags = prm.debug_flags;
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
        int *sptr = reinterpret_cast<int *>(e);
        e += align_up(sizeof(int) * (kMaxBlocks + 1), 256);
        int *rptr = reinterpret_cast<int *>(e);
        e += align_up(sizeof(int) * (kMaxBlocks + 1), 256);
        Segment *ssegs = reinterpret_cast<Segment *>(e);
        e += align_up(sizeof(Segment) * (size_t)(kMaxBlocks + P), 256);
        Segment *rsegs = reinterpret_cast<Segment *>(e);
        std::vector<long long> ct(P), rt(P);
        std::vector<int> cw(P), rw(P, 1);
        for (int p = 0; p < P; ++p) {
            ct[p] = (pds[p].n + kTile - 1) / kTile;
            rt[p] = (pds[p].m + kTile - 1) / kTile;
            cw[p] = pds[p].d;
        }
        std::vector<int> hsp, hrp;
        std::vector<Segment> hss, hrs;
        partition(ct, cw, G, hsp, hss);
        partition(rt, rw, G, hrp, hrs);
        CCS_CUDA_TRY(cudaMemcpyAsync(d_probs, pds.data(), sizeof(ProblemDev) * P,
                                     cudaMemcpyHostToDevice, s));
        CCS_CUDA_TRY(cudaMemcpyAsync(sptr, hsp.data(), sizeof(int) * (G + 1),
                                     cudaMemcpyHostToDevice, s));
        CCS_CUDA_TRY(cudaMemcpyAsync(rptr, hrp.data(), sizeof(int) * (G + 1),
                                     cudaMemcpyHostToDevice, s));
        if (!hss.empty())
            CCS_CUDA_TRY(cudaMemcpyAsync(ssegs, hss.data(), sizeof(Segment) * hss.size(),
                                         cudaMemcpyHostToDevice, s));
        if (!hrs.empty())
            CCS_CUDA_TRY(cudaMemcpyAsync(rsegs, hrs.data(), sizeof(Segment) * hrs.size(),
                                         cudaMemcpyHostToDevice, s));
        a.probs = d_probs;
        a.score_ptr = sptr;
        a.score_segs = ssegs;
        a.res_ptr = rptr;
        a.res_segs = rsegs;
    }

    void *args[] = {&a};
    const int ev = prof_start(CCS_K_PERSISTENT, s);
    CCS_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)fn, dim3(G), dim3(threads), args, smem, s));
    prof_stop(ev, s);
    count_launches(1);
    if (dev_out) return CCS_OK;  // asynchronous: the kernel writes the results

    // results: one copy of the sync word and every control block
    std::vector<char> hdr(sizeof(EngineSync) + sizeof(DecodeCtrl) * (size_t)P);
    CCS_CUDA_TRY(cudaMemcpyAsync(hdr.data(), ws, hdr.size(), cudaMemcpyDeviceToHost, s));
    std::vector<unsigned long long> hst;
    if (a.stamps) {
        hst.resize(kSubBase + 3 * kMaxStampIters);
        CCS_CUDA_TRY(cudaMemcpyAsync(hst.data(), stamps, sizeof(unsigned long long) * hst.size(),
                                     cudaMemcpyDeviceToHost, s));
    }
    CCS_CUDA_TRY(cudaStreamSynchronize(s));
    EngineSync hs;
    std::memcpy(&hs, hdr.data(), sizeof(hs));
    const int herr = hs.error;
    int max_it = 0;
    for (int p = 0; p < P; ++p) {
        DecodeCtrl hc;
        std::memcpy(&hc, hdr.data() + sizeof(EngineSync) + sizeof(DecodeCtrl) * (size_t)p,
                    sizeof(hc));
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

}  // namespace ccs

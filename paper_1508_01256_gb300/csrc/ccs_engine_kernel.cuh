// ccs_engine_kernel.cuh -- Parallel-l0 (Alg. 2) in one persistent cooperative
// launch: the kernel template k_engine<DMAX, THREADS> and its device code.
// Its instances are compiled in ccs_engine_k<threads>_d<pair>.cu (two per
// file, so they build in parallel); ccs_engine.cu plans and launches them.
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
//   - the problem's residual fingerprints (m 16-bit values when m <= 32768,
//     else m bytes) and the segment's
//     CSC row indices stream into shared memory by TMA bulk copies
//     (cp.async.bulk, mbarrier completion); the CSC goes through a ring of
//     stages so the next chunks are in flight while warps work on this one;
//   - each warp tests its 32 columns against the fingerprint bound (a value's
//     count never exceeds its fingerprint's count), from shared memory only:
//     first the zero count, then whether any two nonzero fingerprints are
//     equal, and the full count only when the score needs three or more
//     (columns that pass the zero count are gathered 32 at a time in a
//     per-warp buffer when a tile has few of them);
//   - the few columns that may reach alpha are queued, then scored exactly,
//     lane-parallel across the CTA: d binary64 gathers of r each.
// Problems whose fingerprints do not fit shared memory score every column
// exactly from the same stages.
//
// Every wait (grid barrier, mbarrier) is bounded by the watchdog: on time-out
// the CTA records kErrWatchdog, gives its in-flight copies a bounded time to
// land, and returns; the host reports CCS_ETIMEOUT.
#pragma once

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
constexpr int kFlagOrdered = 2;     // test hook: ordered residual from the start
constexpr int kFlagSwitch = 4;      // test hook: the certificate fails from iteration 2
constexpr int kFlagRowInline = 8;   // test hook: row-driven candidates scored inline, no queue
constexpr int kFlagRowAlways = 16;  // test hook: row-driven whenever the row list fits
constexpr int kFlagRowNever = 32;   // every score phase streams the CSC
constexpr int kFlagStreamInline = 64;  // stream candidates scored where found, not queued
constexpr int kFpChunk = 32768;     // bytes per fingerprint bulk copy
constexpr int kWbufPerWarp = 32;    // buffered candidate columns per consumer warp
// A buffered column's entry: its index, then its fingerprints packed two
// (16-bit) or four (8-bit) to a word, so the buffer's test reads shared
// memory only.
template <int DMAX>
constexpr int kWbufEntry = 1 + (DMAX + 1) / 2;
constexpr int kSubBase = 3 * kMaxStampIters + 2;  // CTA-0 score sub-phase stamps start here
constexpr int kRowDrivenDiv = 64;   // row-driven score phase while ||r||_0 <= m / kRowDrivenDiv
constexpr long long kRowDrivenMinEntries = 64ll << 20;  // ... and the CSC (n d entries) streams
                                                       // from HBM, not from L2
constexpr int kRowUnroll = 16;      // CSR entries in flight per thread in that phase

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
    int shifted;                // 1: the shifted variant (Sec. 4.3.1)
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

__device__ __forceinline__ void red_release_add(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
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

// An L2 policy that marks lines as the first to evict.  The CSC streams
// through L2 once per score phase (604 MB at n = 2^24, d = 9, several times
// the L2); with the default policy it evicts r, the fingerprints and the
// queued candidates' x_hat, whose gathers then wait behind the stream in
// HBM.  Marked evict-first, the stream replaces its own lines first.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// bulk_g2s with an L2 cache policy for the source lines.
__device__ __forceinline__ void bulk_g2s_hint(void *dst, const void *src, uint32_t bytes,
                                              uint64_t *bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
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
static __device__ bool grid_barrier(const EngineArgs &a, unsigned index, bool arrive = true) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        // the CTA barrier above orders every thread's writes before thread 0's
        // release; the acquire polls order the other CTAs' writes before what
        // follows the CTA barrier below
        if (arrive) red_release_add(&a.sync->arrive, 1u);
        const unsigned target = (index + 1u) * gridDim.x;
        const unsigned long long t0 = globaltimer();
        for (unsigned polls = 0; ld_acquire(&a.sync->arrive) < target; ++polls) {
            if ((polls & 15u) == 15u &&
                (*reinterpret_cast<volatile int *>(&a.sync->error) != 0 ||
                 globaltimer() - t0 > (unsigned long long)a.watchdog_ns)) {
                atomicOr(&a.sync->error, kErrWatchdog);
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
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
    // the segment's descriptor is staged in shared memory: the segment's
    // code reads its fields many times, and a.probs lives in global memory
    __shared__ ProblemDev s_seg;
    for (int p = lo; p < a.P && pref[p] < B1; ++p) {
        const ProblemDev &G = problem(a, p);
        if (!part_on(a, G, status[p], kind)) continue;
        const long long w = part_weight(G, kind), tiles = part_tiles(G, kind);
        const long long t0 = B0 > pref[p] ? (B0 - pref[p] + w - 1) / w : 0;
        const long long t1 = min(tiles, (B1 - pref[p] + w - 1) / w);
        if (t1 > t0) {
            __syncthreads();  // the previous segment is done with s_seg
            if (threadIdx.x < (int)(sizeof(ProblemDev) / sizeof(int)))
                reinterpret_cast<int *>(&s_seg)[threadIdx.x] =
                    reinterpret_cast<const int *>(&G)[threadIdx.x];
            __syncthreads();
            fn(p, s_seg, (int)t0, (int)t1);
        }
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
    int *wbuf;         // per consumer warp: kWbufPerWarp buffered candidate columns,
                       // kWbufEntry<DMAX> ints each
    unsigned long long *xmax;  // bits of the largest |x_hat_j| this CTA set (exact mode)
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
    if (tma)
        bulk_g2s_hint(S.stage + (size_t)slot * a.stage_bytes, P.csc_rows + col0 * P.d, tma, bar,
                      l2_evict_first_policy());
}

// Copies a one-problem launch issues ahead of its score phase (thread 0's
// record).  The CSC does not change between iterations and a CTA's segment
// of a lone problem is the same in every iteration, so the first chunks of
// the next score phase can enter the ring before the phase begins, as can
// the fingerprints once the grid barrier after their last store has opened.
struct Prefetch {
    int chunks;  // chunks 0 .. chunks-1 of the next segment are in the ring
    bool fp;     // the next fingerprint copy is in flight
};

// Issue the first chunk of a segment ahead of its score phase (the producer
// issues the rest when the phase begins).  Only one: the fingerprint copy
// issued just before must land before any column can be tested, and a whole
// ring of chunks from HBM would share the SM's bandwidth with it (measured:
// the fingerprint wait drops from ~8 us to ~5 us at n = 2^24).  Thread 0
// only; the ring's previous chunks are all consumed.
__device__ __forceinline__ void prefetch_chunks(const EngineArgs &a, const ProblemDev &P, int lo,
                                                int hi, int per, ScoreSmem &S, unsigned chunk_seq,
                                                Prefetch &pf, bool &ok) {
    const int nchunks = (hi - lo + per - 1) / per;
    const int c1 = min(nchunks, 1);
    for (int c = pf.chunks; c < c1; ++c) {
        const unsigned seq = chunk_seq + c;
        const int slot = seq % a.stages;
        if (!mbar_wait(a, &S.empty[slot], ((seq / a.stages) & 1u) ^ 1u)) {
            ok = false;
            return;
        }
        issue_chunk(a, P, lo, hi, c, per, S, slot);
        pf.chunks = c + 1;
    }
}

// Issue the fingerprint copy of the next score phase.  Thread 0 only, after
// the grid barrier that follows the fingerprints' last generic stores.
__device__ __forceinline__ void prefetch_fp(const ProblemDev &P, ScoreSmem &S, Prefetch &pf) {
    asm volatile("fence.proxy.async.global;" ::: "memory");
    const uint32_t total = (uint32_t)align_up((size_t)P.m * (fp16_for(P.m) ? 2 : 1), 16);
    mbar_expect_tx(S.fp_bar, total);
    for (uint32_t off = 0; off < total; off += kFpChunk)
        bulk_g2s(S.fp + off, P.fp + off, min((uint32_t)kFpChunk, total - off), S.fp_bar);
    pf.fp = true;
}

// Before the CTA leaves: wait (bounded) for the copies issued ahead, which
// no score phase will consume.  Thread 0 only.
__device__ __forceinline__ void drain_prefetch(const EngineArgs &a, ScoreSmem &S,
                                               unsigned chunk_seq, unsigned fp_seq, Prefetch &pf) {
    for (int c = 0; c < pf.chunks; ++c) {
        const unsigned seq = chunk_seq + c;
        if (!mbar_wait(a, &S.full[seq % a.stages], (seq / a.stages) & 1u)) break;
    }
    if (pf.fp) mbar_wait(a, S.fp_bar, fp_seq & 1u);
    pf.chunks = 0;
    pf.fp = false;
}

// Exact score and apply of one column inside the stream, from its rows in
// registers.  kCandidate: the column passed the fingerprint test (the queue
// was full), so it is likely accepted: x_hat_j and the in-slots flag are
// loaded in the same round as the r gathers.  Otherwise (problems without
// shared-memory fingerprints) most columns are rejected: kPrefilter applies
// the fingerprint bound of the gathered values before the O(d^2) compare,
// and x_hat_j is loaded only for accepted columns.
template <int DMAX, bool kPrefilter, bool kCandidate>
__device__ __forceinline__ bool score_inline(const EngineArgs &a, const ProblemDev &P, int j,
                                             const int32_t (&rows)[DMAX], bool exact,
                                             unsigned long long *xmax_s, int spos) {
    const int d = P.d;
    unsigned long long v[DMAX];
#pragma unroll
    for (int t = 0; t < DMAX; ++t) v[t] = (t < d) ? value_bits(__ldcg(P.r + rows[t])) : 0ull;
    double xj = 0.0;
    uint8_t ins = 1;
    if (kCandidate) {
        xj = __ldcg(P.x_hat + j);
        if (!exact) ins = __ldcg(P.in_slots + j);
    }
    unsigned long long omega;
    bool acc;
    if (spos >= 0) {
        acc = exact_score_shifted<DMAX>(v, d, spos, a.alpha, a.mode, &omega);
    } else {
        if (kPrefilter && !values_may_accept<DMAX>(v, d, a.alpha, a.mode)) return false;
        acc = exact_score_values<DMAX>(v, d, a.alpha, a.mode, &omega);
    }
    if (acc) {
        if (!kCandidate) {
            xj = __ldcg(P.x_hat + j);
            if (!exact) ins = __ldcg(P.in_slots + j);
        }
        if (exact) apply_exact<DMAX>(P, j, rows, d, omega, xj, xmax_s);
        else apply_pair_loaded<DMAX>(P, j, rows, d, omega, xj, ins);
    }
    return acc;
}

// Queued candidates: exact score, lane-parallel over the CTA.  The r
// gathers, x_hat_j and the in-slots flag go out in one round trip.
template <int DMAX>
__device__ __forceinline__ void score_queue(const EngineArgs &a, const ProblemDev &P,
                                         const int32_t *queue, int qn,
                                         unsigned long long *acc_smem, bool ok, bool exact,
                                         unsigned long long *xmax_s, int spos) {
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
            const uint8_t ins = exact ? (uint8_t)0 : __ldcg(P.in_slots + j);
            unsigned long long omega;
            acc = (spos >= 0) ? exact_score_shifted<DMAX>(v, d, spos, a.alpha, a.mode, &omega)
                              : exact_score_values<DMAX>(v, d, a.alpha, a.mode, &omega);
            if (acc) {
                if (exact) apply_exact<DMAX>(P, j, rows, d, omega, xj, xmax_s);
                else apply_pair_loaded<DMAX>(P, j, rows, d, omega, xj, ins);
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, acc);
        if (lane == 0 && bal) atomicAdd(acc_smem, (unsigned long long)__popc(bal));
    }
}

// Once r is sparse few columns pass the zero count.  A warp with fewer than
// kDenseLanes such lanes in a tile does not test them there: it appends them
// to its buffer and tests them 32 at a time, so the rest of the test runs on
// full warps instead of once per tile that has a passing lane.  The
// 1024-thread instance (64 registers a thread) always tests in place: there
// the buffer path costs more in spills than it saves (measured at n=2^20,
// m=2^17 and at n=2^24, m=16777, both d=7; at d=9 on 512 threads it saves 5 %).
constexpr int kDenseLanes = 12;
template <int THREADS, bool kWide>
constexpr bool kUseWarpBuffer = THREADS != 1024;

// The rest of the fingerprint bound for a column that passed the zero count
// (its fingerprints f, nz of them nonzero): a nonzero pair, then, only when
// the score needs three or more equal values, the full count.
template <int DMAX, bool kWide>
__device__ __forceinline__ bool fp_bound_passes(const unsigned (&f)[DMAX], int d, int need) {
    if (!fp_pair_exists<DMAX>(f, d)) return false;
    return need <= 2 || fp_max_count<DMAX, kWide>(f, d) >= need;
}

// Queue column j (rows in `rows`) for the exact score, or score it inline
// when the queue is full; returns whether it was accepted inline.
template <int DMAX, int THREADS>
__device__ __forceinline__ bool queue_or_score(const EngineArgs &a, const ProblemDev &P,
                                               int32_t *queue, int *qn, int j,
                                               const int32_t (&rows)[DMAX], bool exact,
                                               unsigned long long *xmax_s, int spos) {
    const int q = (a.debug_flags & kFlagStreamInline) ? a.queue_cap : atomicAdd(qn, 1);
    if (q < a.queue_cap) {  // scored after the stream
        int32_t *e = queue + q * (DMAX + 1);
        e[0] = j;
        // x_hat_j is read when the queue is scored: bring its line into L2 now
        asm volatile("prefetch.global.L2 [%0];" ::"l"(P.x_hat + j));
#pragma unroll
        for (int t = 0; t < DMAX; ++t) e[1 + t] = rows[t];
        return false;
    }
    return score_inline<DMAX, false, true>(a, P, j, rows, exact, xmax_s, spos);
}

// Store a column that passed the zero count in entry `slot` of its warp's
// buffer: the index and the packed fingerprints.
template <int DMAX, bool kWide>
__device__ __forceinline__ void wbuf_put(int *wb, int slot, int j, const unsigned (&f)[DMAX]) {
    int *e = wb + slot * kWbufEntry<DMAX>;
    e[0] = j;
    constexpr int kPer = kWide ? 2 : 4, kBits = kWide ? 16 : 8;
#pragma unroll
    for (int q = 0; q < (DMAX + kPer - 1) / kPer; ++q) {
        unsigned w = 0u;
#pragma unroll
        for (int t = q * kPer; t < DMAX && t < (q + 1) * kPer; ++t) w |= f[t] << (kBits * (t - q * kPer));
        e[1 + q] = (int)w;
    }
}

// The rest of the fingerprint test, then queue (or inline exact score), of
// up to 32 buffered columns (one per lane), from their packed fingerprints
// in shared memory; only the columns that pass load their rows (from L2,
// shortly after the stream brought them).  Returns the number accepted
// inline.
template <int DMAX, int THREADS, bool kExactD, bool kWide>
__device__ __noinline__ int flush_candidates(const EngineArgs &a, const ProblemDev &P,
                                             int32_t *queue, int *qn, const int *wb, int cnt,
                                             bool exact, unsigned long long *xmax_s) {
    const int lane = threadIdx.x & 31;
    const int d = kExactD ? DMAX : P.d;
    bool acc = false;
    if (lane < cnt) {
        const int *e = wb + lane * kWbufEntry<DMAX>;
        const int j = e[0];
        constexpr int kPer = kWide ? 2 : 4, kBits = kWide ? 16 : 8;
        constexpr unsigned kMask = kWide ? 0xffffu : 0xffu;
        unsigned f[DMAX];
        int nz = 0;
#pragma unroll
        for (int t = 0; t < DMAX; ++t) {
            f[t] = (t < d) ? ((unsigned)e[1 + t / kPer] >> (kBits * (t % kPer))) & kMask : 0u;
            nz += (f[t] != 0u);
        }
        const int need = (a.mode == CCS_SCORE_COUNT) ? a.alpha : a.alpha + (d - nz);
        if (fp_bound_passes<DMAX, kWide>(f, d, need)) {
            int32_t rows[DMAX];
#pragma unroll
            for (int t = 0; t < DMAX; ++t) rows[t] = (t < d) ? __ldg(P.csc_rows + (size_t)j * d + t) : 0;
            acc = queue_or_score<DMAX, THREADS>(a, P, queue, qn, j, rows, exact, xmax_s, -1);
        }
    }
    return __popc(__ballot_sync(0xffffffffu, acc));
}

// Consumer side of the score phase for one segment (warps 1..): wait for
// each chunk, test its columns, release the stage.  kExactD: d == DMAX, so
// every loop over a column's rows has a compile-time trip count.  kWide:
// the problem keeps 16-bit fingerprints.
template <int DMAX, int THREADS, bool kExactD, bool kWide>
__device__ __forceinline__ void consume_segment(const EngineArgs &a, const ProblemDev &P,
                                                const Segment &sg, int per, int nchunks,
                                                unsigned chunk_seq, ScoreSmem &S, int *wb,
                                                bool exact, int spos, bool zero_x, bool &ok) {
    constexpr int kTpw = (THREADS == 512) ? 2 : 1;
    const int warps = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int d = kExactD ? DMAX : P.d;
    const bool use_fp = (P.flags & kPdUseFp) != 0;
    const unsigned lt_mask = (1u << lane) - 1u;
    int wbn = 0;     // buffered columns of this warp (warp-uniform)
    int n_acc = 0;   // columns accepted by the buffer flushes (warp-uniform)
    int n_mine = 0;  // columns this lane accepted inline
    // ring slot and phase of chunk c, advanced by one per chunk (no division
    // in the loop)
    int slot = (int)(chunk_seq % (unsigned)a.stages);
    unsigned phase = (chunk_seq / (unsigned)a.stages) & 1u;
    for (int c = 0; c < nchunks; ++c, slot = (slot + 1 == a.stages) ? (phase ^= 1u, 0) : slot + 1) {
        ok = ok && mbar_wait(a, &S.full[slot], phase);
        ok = __all_sync(0xffffffffu, ok);  // warp-uniform: the tile loop votes
        const int32_t *stage = reinterpret_cast<const int32_t *>(S.stage + (size_t)slot * a.stage_bytes);
        long long col0, col1;
        chunk_cols(P, sg.lo, sg.hi, c, per, col0, col1);
        // ints of this chunk that came by TMA; only a problem's last chunk
        // can end with up to 3 ints that did not
        const int ncol = (int)(col1 - col0);  // at most (warps - 1) * kTpw * 32
        const int e_tma = ((ncol * d * 4) & ~15) / 4;
        const bool tail = e_tma != ncol * d;
#pragma unroll
        for (int u = 0; u < kTpw; ++u) {
            const int tile = sg.lo + c * per + u * (warps - 1) + (warp - 1);
            if (!ok || tile >= sg.hi) continue;  // warp-uniform
            const int base = tile * kTile;
            const bool live = lane < P.n - base;
            const int j = base + lane;
            // first score phase of a lone problem: x_hat <- 0 (Alg. 2's first
            // line) is stored here, one coalesced line a tile, while the
            // stream has bandwidth to spare, instead of in a pass of its own;
            // every later read of x_hat_j follows this store in the same
            // thread, after a __syncwarp (buffered columns) or after a
            // __syncthreads (queued columns)
            if (zero_x && live) P.x_hat[j] = 0.0;
            const int e0 = (j - (int)col0) * d;  // first int of column j in the stage
            int32_t rows[DMAX];
            if (!tail) {
#pragma unroll
                for (int t = 0; t < DMAX; ++t) rows[t] = (t < d && live) ? stage[e0 + t] : 0;
            } else {
#pragma unroll
                for (int t = 0; t < DMAX; ++t)
                    rows[t] = (t < d && live) ? ((e0 + t < e_tma) ? stage[e0 + t]
                                                                  : __ldg(P.csc_rows + (size_t)j * d + t))
                                              : 0;
            }
            bool acc = false;
            if (!use_fp) {
                if (live)
                    acc = score_inline<DMAX, THREADS != 1024, false>(a, P, j, rows, exact, S.xmax,
                                                                     spos);
            } else {
                // the fingerprint bound: enough nonzero rows for the score
                // (zero count), then a nonzero pair, then, only when the
                // score needs three or more equal values, the full count
                unsigned f[DMAX];
                int nz = 0;
#pragma unroll
                for (int t = 0; t < DMAX; ++t) {
                    f[t] = (t < d) ? fp_at<kWide>(S.fp, rows[t]) : 0u;
                    nz += (f[t] != 0u);
                }
                const int need = (a.mode == CCS_SCORE_COUNT) ? a.alpha : a.alpha + (d - nz);
                if (spos >= 0) {
                    // shifted: the candidate's fingerprint count bounds its count
                    unsigned fw = 0u;
#pragma unroll
                    for (int t = 0; t < DMAX; ++t) fw = (t == spos) ? f[t] : fw;
                    int cf = 0;
#pragma unroll
                    for (int t = 0; t < DMAX; ++t) cf += (t < d) & (f[t] == fw);
                    if (live && fw != 0u && nz >= need && cf >= need)
                        acc = queue_or_score<DMAX, THREADS>(a, P, S.queue, S.qn, j, rows, exact,
                                                            S.xmax, spos);
                    n_mine += acc;
                    continue;
                }
                const bool pass = live && nz >= need;
                const unsigned bal = __ballot_sync(0xffffffffu, pass);
                if (bal) {
                    if (!kUseWarpBuffer<THREADS, kWide> || __popc(bal) >= kDenseLanes) {
                        if (pass && fp_bound_passes<DMAX, kWide>(f, d, need))
                            acc = queue_or_score<DMAX, THREADS>(a, P, S.queue, S.qn, j, rows,
                                                                exact, S.xmax, -1);
                    } else if constexpr (kUseWarpBuffer<THREADS, kWide>) {
                        // append; a full buffer is tested right away and the
                        // lanes that did not fit start the next one
                        const int cnt = __popc(bal);
                        const int slot_w = wbn + __popc(bal & lt_mask);
                        if (pass && slot_w < 32) wbuf_put<DMAX, kWide>(wb, slot_w, j, f);
                        if (wbn + cnt >= 32) {
                            __syncwarp();
                            n_acc += flush_candidates<DMAX, THREADS, kExactD, kWide>(
                                a, P, S.queue, S.qn, wb, 32, exact, S.xmax);
                            __syncwarp();
                            if (pass && slot_w >= 32) wbuf_put<DMAX, kWide>(wb, slot_w - 32, j, f);
                            wbn += cnt - 32;
                        } else {
                            wbn += cnt;
                        }
                    }
                }
            }
            n_mine += acc;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.empty[slot]);  // this warp is done with the stage
    }
    if (kUseWarpBuffer<THREADS, kWide> && wbn > 0 && ok) {
        __syncwarp();
        n_acc += flush_candidates<DMAX, THREADS, kExactD, kWide>(a, P, S.queue, S.qn, wb, wbn,
                                                                 exact, S.xmax);
    }
    n_acc += (int)__reduce_add_sync(0xffffffffu, (unsigned)n_mine);
    if (lane == 0 && n_acc) atomicAdd(S.acc, (unsigned long long)n_acc);
}

// Score phase of one segment.  Warp 0 is the producer: its lane 0 streams
// the fingerprints and the CSC chunks by TMA, refilling a stage as soon as
// every consumer warp has released it.  Warps 1.. consume their tiles of
// each chunk (consume_segment).  Then every warp scores the queued
// candidates exactly.
//
// rmode: 0 while the problem's incremental residual is certified exact
// (accepted pairs update r_next by atomic adds), 1 for the ordered residual
// (contributor records), 2 in the iteration that switches from 0 to 1 (the
// segment's nonzero columns enter their rows' records first).  it: the
// problem's own iteration number.
// Switch of a segment to the ordered residual: its columns that are already
// nonzero enter their rows' contributor records, and every column's in-slots
// flag is set from x_hat (r itself is exact and current, so no row is marked
// touched).
// x_zero: x_hat is known to be zero (it is not read: the first score phase of
// a lone problem has not stored it yet).
template <int DMAX>
__device__ __forceinline__ void enter_segment_slots(const ProblemDev &P, int seg_lo, int seg_hi,
                                                    bool x_zero = false) {
    const long long c1 = min((long long)P.n, (long long)seg_hi * kTile);
    for (long long j = (long long)seg_lo * kTile + threadIdx.x; j < c1; j += blockDim.x) {
        const bool nz = !x_zero && __ldcg(P.x_hat + j) != 0.0;
        P.in_slots[j] = nz ? 1 : 0;
        if (nz) {
            int32_t rows[DMAX];
#pragma unroll
            for (int t = 0; t < DMAX; ++t)
                rows[t] = (t < P.d) ? __ldg(P.csc_rows + (size_t)j * P.d + t) : 0;
            enter_slots<DMAX>(P, (int)j, rows, P.d);
        }
    }
}

template <int DMAX, int THREADS>
__device__ __forceinline__ void score_segment(const EngineArgs &a, const ProblemDev &P,
                                              int seg_lo, int seg_hi, int g, int it, int rmode,
                                              ScoreSmem &S, unsigned &chunk_seq,
                                              unsigned &fp_seq, bool &ok,
                                              Prefetch *pf = nullptr, bool zero_x = false) {
    const bool exact = rmode == 0;
    const int spos = a.shifted ? it % P.d : -1;  // shifted variant: candidate row
    const Segment sg{0, seg_lo, seg_hi, 0};
    const int warps = blockDim.x >> 5;
    constexpr int kTpw = (THREADS == 512) ? 2 : 1;  // tiles per consumer warp and chunk
    const int per = (warps - 1) * kTpw;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool use_fp = (P.flags & kPdUseFp) != 0;
    const int tiles = sg.hi - sg.lo;
    const int nchunks = (tiles + per - 1) / per;
    unsigned long long *acc_slot = &P.ctrl->acc[g & 3];

    __syncthreads();  // previous users of the queue and fingerprints are done
    if (threadIdx.x == 0) {
        *S.qn = 0;
        *S.acc = 0;
        *S.xmax = 0;
    }
    if (rmode == 2) enter_segment_slots<DMAX>(P, seg_lo, seg_hi, zero_x);
    __syncthreads();

    if (warp == 0) {
        if (lane == 0 && ok) {
            if (use_fp && !(pf && pf->fp)) {
                // the fingerprints were written by generic stores (residual
                // phase, any SM) before the grid barrier; order them before
                // this thread's bulk (async-proxy) reads
                asm volatile("fence.proxy.async.global;" ::: "memory");
                const uint32_t total =
                    (uint32_t)align_up((size_t)P.m * (fp16_for(P.m) ? 2 : 1), 16);
                mbar_expect_tx(S.fp_bar, total);
                for (uint32_t off = 0; off < total; off += kFpChunk)
                    bulk_g2s(S.fp + off, P.fp + off, min((uint32_t)kFpChunk, total - off), S.fp_bar);
            }
            const int c0 = pf ? pf->chunks : 0;
            int slot = (int)((chunk_seq + c0) % (unsigned)a.stages);
            unsigned phase = ((chunk_seq + c0) / (unsigned)a.stages) & 1u;
            for (int c = c0; c < nchunks;
                 ++c, slot = (slot + 1 == a.stages) ? (phase ^= 1u, 0) : slot + 1) {
                if (!mbar_wait(a, &S.empty[slot], phase ^ 1u)) {
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
        int *wb = S.wbuf + (warp - 1) * kWbufPerWarp * kWbufEntry<DMAX>;
        const bool wide = fp16_for(P.m);
        if (P.d == DMAX) {
            if (wide)
                consume_segment<DMAX, THREADS, true, true>(a, P, sg, per, nchunks, chunk_seq, S, wb, exact, spos, zero_x, ok);
            else
                consume_segment<DMAX, THREADS, true, false>(a, P, sg, per, nchunks, chunk_seq, S, wb, exact, spos, zero_x, ok);
        } else {
            if (wide)
                consume_segment<DMAX, THREADS, false, true>(a, P, sg, per, nchunks, chunk_seq, S, wb, exact, spos, zero_x, ok);
            else
                consume_segment<DMAX, THREADS, false, false>(a, P, sg, per, nchunks, chunk_seq, S, wb, exact, spos, zero_x, ok);
        }
    }
    chunk_seq += nchunks;
    if (use_fp) ++fp_seq;
    if (pf && threadIdx.x == 0) {
        pf->chunks = 0;  // taken by this segment (thread 0 is its producer)
        pf->fp = false;
    }
    __syncthreads();  // stream done, queue complete
    if (a.stamps && blockIdx.x == 0 && threadIdx.x == 0 && g < kMaxStampIters)
        a.stamps[kSubBase + 3 * g + 1] = globaltimer();

    score_queue<DMAX>(a, P, S.queue, min(*S.qn, a.queue_cap), S.acc, ok, exact, S.xmax, spos);
    // one global atomic per CTA and segment (all warps' counts summed on chip)
    __syncthreads();
    if (threadIdx.x == 0) {
        if (*S.acc) atomicAdd(acc_slot, *S.acc);
        if (exact && *S.xmax) atomicMax(&P.ctrl->xmax[(it + 1) & 1], *S.xmax);
        if (a.stamps && blockIdx.x == 0 && g < kMaxStampIters)
            a.stamps[kSubBase + 3 * g + 2] = globaltimer();
    }
}

// ---- row-driven score phase (one problem per launch, small ||r||_0) ---------
//
// A column can be accepted only if at least T of its d rows hold a nonzero
// r_i: its l0 decrease (Eq. 15) is at most (nonzero rows) - (zero rows), so
// T = ceil((alpha + d) / 2); its match count (Alg. 8) is at most the nonzero
// rows, so T = alpha.  Once ||r||_0 is small, the columns that reach T are
// found from the CSR rows of the nonzero r_i -- the CTAs split those rows'
// entries evenly and count each column's hits in a byte per column -- and
// only they are scored exactly, as the column stream would score them.
// Every other column keeps a score below alpha, so the accepted set, and the
// decode, are the ones of the column stream, bit for bit.  The phase reads
// the CSR entries of the nonzero rows (||r||_0 * nd/m on average) instead of
// the whole CSC (4dn bytes).

// Which score phase iteration `it` of a lone problem takes.  Every CTA
// evaluates it from the same stored ||r||_0, so all agree.  The row list
// lives in the CSC stage ring (16 bytes a row).  Measured on a GB300, a CSR
// entry counted by a global atomic costs 35-60 times a column entry of the
// CSC stream, so the phase pays only while ||r||_0 is a few percent of m,
// and only when the stream comes from HBM (an L2-resident CSC streams too
// fast for the phase's fixed cost to pay back).
__device__ __forceinline__ bool row_driven_iter(const EngineArgs &a, const ProblemDev &P, int it,
                                                long long r0) {
    if (a.probs || !(P.flags & kPdUseFp) || it < 1 || r0 <= 0 || (a.debug_flags & kFlagRowNever))
        return false;
    const long long cap = ((long long)a.stages * a.stage_bytes - 16) / 16;
    return r0 <= cap && ((a.debug_flags & kFlagRowAlways) ||
                         (r0 * kRowDrivenDiv <= (long long)P.m &&
                          (long long)P.n * P.d >= kRowDrivenMinEntries));
}

// Row list of a row-driven phase in the stage ring: the nonzero rows in
// ascending order, the CSR offset of each, and the exclusive prefix of their
// degrees (pref[R] = E, the entries of all of them).
struct RowList {
    long long *ptr0;  // cap
    int *pref;        // cap + 1
    int *rows;        // cap
};

__device__ __forceinline__ RowList row_list(const EngineArgs &a, const ScoreSmem &S) {
    const int cap = (int)(((long long)a.stages * a.stage_bytes - 16) / 16);
    RowList L;
    L.ptr0 = reinterpret_cast<long long *>(S.stage);
    L.pref = reinterpret_cast<int *>(L.ptr0 + cap);
    L.rows = L.pref + cap + 1;
    return L;
}

// Block-wide exclusive prefix of one int per thread; *total gets the sum.
template <int THREADS>
__device__ __noinline__ int block_excl_scan(int v, int *total) {
    __shared__ int s_w[THREADS / 32];
    __shared__ int s_tot;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    __syncthreads();  // earlier users of s_w are done
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += s_w[w];
    if (threadIdx.x == THREADS - 1) s_tot = before + inc;
    __syncthreads();
    *total = s_tot;
    return before + inc - v;
}

// Nonzero fingerprints in a 32-bit word of the array (2 of 16 bits or 4 of
// 8 bits); bit t of the mask: entry t of the word.
template <bool kWide>
__device__ __forceinline__ unsigned fp_word_mask(unsigned w) {
    if constexpr (kWide) return ((w & 0xffffu) != 0u) | (((w >> 16) != 0u) << 1);
    else
        return ((w & 0xffu) != 0u) | ((((w >> 8) & 0xffu) != 0u) << 1) |
               ((((w >> 16) & 0xffu) != 0u) << 2) | (((w >> 24) != 0u) << 3);
}

// Fill the row list from the fingerprints in shared memory (fp_i == 0 iff
// r_i == 0).  Each warp takes a contiguous run of 32-bit words and its lanes
// read consecutive words (no bank conflicts); a first pass counts, a block
// scan places the warps, a second pass writes the rows in ascending order.
// Returns R (every CTA builds the same list); *E the entries.
template <int THREADS, bool kWide>
__device__ __forceinline__ int list_nonzero_rows(const ProblemDev &P, const uint8_t *fp,
                                                 const RowList &L, int cap, int *E) {
    constexpr int kW = THREADS / 32, kPer = kWide ? 2 : 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned *fw = reinterpret_cast<const unsigned *>(fp);
    const int nw = (P.m + kPer - 1) / kPer;  // words; entries past row m - 1 are masked
    const unsigned last = (P.m % kPer) ? (1u << (P.m % kPer)) - 1u : (1u << kPer) - 1u;
    const int w0 = (int)((long long)nw * warp / kW), w1 = (int)((long long)nw * (warp + 1) / kW);
    auto word_mask = [&](int w) {
        const unsigned msk = fp_word_mask<kWide>(fw[w]);
        return w == nw - 1 ? msk & last : msk;
    };
    int cnt = 0;
    for (int w = w0 + lane; w < w1; w += 32) cnt += __popc(word_mask(w));
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    int R;
    int base = block_excl_scan<THREADS>(lane == 0 ? cnt : 0, &R);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int w0r = w0; w0r < w1; w0r += 32) {
        const int w = w0r + lane;
        const unsigned msk = w < w1 ? word_mask(w) : 0u;
        const int c = __popc(msk);
        int inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        int k = base + inc - c;
        for (unsigned b = msk; b; b &= b - 1) {
            const int i = w * kPer + __ffs(b) - 1;
            if (k < cap) L.rows[k] = i;
            ++k;
        }
        base += __shfl_sync(0xffffffffu, inc, 31);
    }
    R = min(R, cap);  // R == ||r||_0 <= cap by row_driven_iter
    __syncthreads();
    const int per2 = (R + THREADS - 1) / THREADS;
    const int q0 = min(R, (int)threadIdx.x * per2), q1 = min(R, q0 + per2);
    int sum = 0;
    for (int q = q0; q < q1; ++q) {
        const int i = L.rows[q];
        const long long p0 = __ldg(P.csr_ptr + i), p1 = __ldg(P.csr_ptr + i + 1);
        L.ptr0[q] = p0;
        L.pref[q] = (int)(p1 - p0);  // degree for now
        sum += (int)(p1 - p0);
    }
    int off = block_excl_scan<THREADS>(sum, E);
    for (int q = q0; q < q1; ++q) {
        const int deg = L.pref[q];
        L.pref[q] = off;
        off += deg;
    }
    if (threadIdx.x == 0) L.pref[R] = *E;
    __syncthreads();
    return R;
}

// This CTA's share [lo, hi) of the E entries, and the row holding entry f.
__device__ __forceinline__ void row_share(long long E, long long &lo, long long &hi) {
    lo = E * blockIdx.x / gridDim.x;
    hi = E * (blockIdx.x + 1) / gridDim.x;
}

__device__ __forceinline__ int row_of_entry(const RowList &L, int R, long long f) {
    int lo = 0, hi = R - 1;  // last q with pref[q] <= f
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (L.pref[mid] <= f) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Visit this CTA's entries: each warp takes a contiguous part of the CTA's
// share and its lanes read consecutive entries (coalesced), kRowUnroll per
// lane at a time; fn(cols) gets those column indices (-1 where none),
// loaded together.  A lane's row cursor moves forward only.
template <int THREADS, typename F>
__device__ __forceinline__ void for_my_row_entries(const ProblemDev &P, const RowList &L, int R,
                                                   long long E, F &&fn) {
    long long lo, hi;
    row_share(E, lo, hi);
    if (hi <= lo || R == 0) return;
    constexpr int kW = THREADS / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long wlo = lo + (hi - lo) * warp / kW, whi = lo + (hi - lo) * (warp + 1) / kW;
    if (whi <= wlo) return;
    long long f0 = wlo + lane;
    int q = row_of_entry(L, R, f0 < whi ? f0 : wlo);
    for (; f0 < whi; f0 += 32LL * kRowUnroll) {
        int cols[kRowUnroll];
#pragma unroll
        for (int u = 0; u < kRowUnroll; ++u) {
            const long long f = f0 + 32LL * u;
            cols[u] = -1;
            if (f < whi) {
                while (L.pref[q + 1] <= f) ++q;
                cols[u] = __ldg(P.csr_cols + L.ptr0[q] + (f - L.pref[q]));
            }
        }
        fn(cols);
    }
}

// Exact score of queued columns (their rows loaded from the CSC first),
// lane-parallel over the CTA; accepted pairs applied as in the stream.
template <int DMAX>
__device__ __forceinline__ void score_queue_cols(const EngineArgs &a, const ProblemDev &P,
                                                 const int32_t *queue, int qn,
                                                 unsigned long long *acc_smem, bool ok,
                                                 bool exact, unsigned long long *xmax_s,
                                                 int spos) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int b0 = warp * 32; b0 < qn; b0 += blockDim.x) {
        const int idx = b0 + lane;
        bool acc = false;
        if (ok && idx < qn) {
            const int j = queue[idx * (DMAX + 1)];
            int32_t rows[DMAX];
#pragma unroll
            for (int t = 0; t < DMAX; ++t)
                rows[t] = (t < P.d) ? __ldg(P.csc_rows + (size_t)j * P.d + t) : 0;
            acc = score_inline<DMAX, false, true>(a, P, j, rows, exact, xmax_s, spos);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, acc);
        if (lane == 0 && bal) atomicAdd(acc_smem, (unsigned long long)__popc(bal));
    }
}

// Out of line (its registers do not add to the column stream's); returns
// the launch's ok flag, and the caller advances the fingerprint sequence.
template <int DMAX, int THREADS>
__device__ __noinline__ bool score_rows(const EngineArgs &a, const ProblemDev &P, int seg_lo,
                                        int seg_hi, int g, int it, int rmode, ScoreSmem S,
                                        unsigned fp_seq, bool ok, Prefetch *pf, int *s_R,
                                        int *s_E) {
    const bool exact = rmode == 0;
    const int spos = a.shifted ? it % P.d : -1;
    const int T = (a.mode == CCS_SCORE_COUNT) ? a.alpha : (a.alpha + P.d + 1) / 2;
    unsigned long long *acc_slot = &P.ctrl->acc[g & 3];
    const RowList L = row_list(a, S);
    const int cap = (int)(((long long)a.stages * a.stage_bytes - 16) / 16);

    __syncthreads();  // previous users of the queue and fingerprints are done
    if (threadIdx.x == 0) {
        *S.qn = 0;
        *S.acc = 0;
        *S.xmax = 0;
    }
    if (rmode == 2) enter_segment_slots<DMAX>(P, seg_lo, seg_hi);
    __syncthreads();
    if (threadIdx.x == 0 && ok && !(pf && pf->fp)) {
        asm volatile("fence.proxy.async.global;" ::: "memory");
        const uint32_t total = (uint32_t)align_up((size_t)P.m * (fp16_for(P.m) ? 2 : 1), 16);
        mbar_expect_tx(S.fp_bar, total);
        for (uint32_t off = 0; off < total; off += kFpChunk)
            bulk_g2s(S.fp + off, P.fp + off, min((uint32_t)kFpChunk, total - off), S.fp_bar);
    }
    ok = ok && mbar_wait(a, S.fp_bar, fp_seq & 1u);
    if (pf && threadIdx.x == 0) pf->fp = false;
    if (!__syncthreads_and(ok)) return false;
    if (a.stamps && blockIdx.x == 0 && threadIdx.x == 0 && g < kMaxStampIters)
        a.stamps[kSubBase + 3 * g] = globaltimer();

    int E = 0;
    const int R = fp16_for(P.m) ? list_nonzero_rows<THREADS, true>(P, S.fp, L, cap, &E)
                                : list_nonzero_rows<THREADS, false>(P, S.fp, L, cap, &E);
    if (threadIdx.x == 0) {
        *s_R = R;
        *s_E = E;
    }
    // count each column's nonzero rows; a column reaching T is a candidate
    unsigned n_inline = 0;
    for_my_row_entries<THREADS>(P, L, R, E, [&](const int (&cols)[kRowUnroll]) {
        unsigned old[kRowUnroll];
#pragma unroll
        for (int u = 0; u < kRowUnroll; ++u)
            old[u] = cols[u] >= 0 ? atomicAdd(P.hits + (cols[u] >> 2), 1u << ((cols[u] & 3) * 8))
                                  : 0u;
#pragma unroll
        for (int u = 0; u < kRowUnroll; ++u) {
            if (cols[u] < 0) continue;
            const unsigned c = (old[u] >> ((cols[u] & 3) * 8)) & 0xffu;
            if (c + 1u != (unsigned)T) continue;
            const int q = (a.debug_flags & kFlagRowInline) ? a.queue_cap : atomicAdd(S.qn, 1);
            if (q < a.queue_cap) {
                S.queue[q * (DMAX + 1)] = cols[u];
                asm volatile("prefetch.global.L2 [%0];" ::"l"(P.csc_rows + (size_t)cols[u] * P.d));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(P.x_hat + cols[u]));
            } else {  // queue full: score it here
                int32_t rows[DMAX];
#pragma unroll
                for (int t = 0; t < DMAX; ++t)
                    rows[t] = (t < P.d) ? __ldg(P.csc_rows + (size_t)cols[u] * P.d + t) : 0;
                n_inline += score_inline<DMAX, false, true>(a, P, cols[u], rows, exact, S.xmax,
                                                            spos);
            }
        }
    });
    if (n_inline) atomicAdd(S.acc, (unsigned long long)n_inline);
    __syncthreads();  // counting done, queue complete
    if (a.stamps && blockIdx.x == 0 && threadIdx.x == 0 && g < kMaxStampIters)
        a.stamps[kSubBase + 3 * g + 1] = globaltimer();
    score_queue_cols<DMAX>(a, P, S.queue, min(*S.qn, a.queue_cap), S.acc, ok, exact, S.xmax,
                           spos);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (*S.acc) atomicAdd(acc_slot, *S.acc);
        if (exact && *S.xmax) atomicMax(&P.ctrl->xmax[(it + 1) & 1], *S.xmax);
        if (blockIdx.x == 0) {
            P.ctrl->row_driven += 1;
            P.ctrl->row_entries += E;
        }
        if (a.stamps && blockIdx.x == 0 && g < kMaxStampIters)
            a.stamps[kSubBase + 3 * g + 2] = globaltimer();
    }
    return ok;
}

// After a row-driven score phase (its counting done on every CTA): every
// counter back to zero.  A coalesced sweep over this CTA's share of the
// n / 4 words (16 bytes a thread and step) costs less than clearing the
// counted words one by one: those are scattered, n / 4 words are few.
template <int THREADS>
__device__ __noinline__ void row_hits_clear(const ProblemDev &P) {
    const long long nw = (P.n + 3) / 4, nq = nw / 4;  // words, whole 16-byte groups
    const long long q0 = nq * blockIdx.x / gridDim.x, q1 = nq * (blockIdx.x + 1) / gridDim.x;
    uint4 *h4 = reinterpret_cast<uint4 *>(P.hits);  // 256-byte aligned in the workspace
    for (long long q = q0 + threadIdx.x; q < q1; q += THREADS) h4[q] = make_uint4(0u, 0u, 0u, 0u);
    if (blockIdx.x == gridDim.x - 1)
        for (long long w = nq * 4 + threadIdx.x; w < nw; w += THREADS) P.hits[w] = 0u;
}

// ---- exactness certificate of the incremental residual --------------------
//
// While every value the method forms -- y_i, r_i, x_hat_j, omega, and every
// partial sum of a row -- is an integer multiple of 2^e (e: the lowest set
// bit over the nonzero y_i) and below 2^(e+53) in magnitude, every binary64
// addition and subtraction of the decode is exact.  Then the ordered row sum
// of Alg. 2's residual equals the sum in any order, and r can be kept by
// subtracting each accepted omega from its column's rows as it is accepted.
// By induction all values stay on the grid of y (omega is a value of r,
// x_hat_j a sum of omegas); the magnitudes at iteration t are bounded by
//   |y_i| + deg * (max|x_hat| + 2 max|r|)
// (a row's partial sums of x_hat, and r_i minus the omegas accepted in its
// row during the iteration).  The test below asks for that bound to stay
// under 2^(e+51), a factor 4 below the limit, which covers the rounding of
// the bound's own evaluation.  Every CTA evaluates it from the same stored
// maxima (written before the previous grid barrier), so all agree.
__device__ __forceinline__ bool exact_certified(const DecodeCtrl *c, int it, int debug_flags) {
    if ((debug_flags & kFlagOrdered) || ((debug_flags & kFlagSwitch) && it >= 2)) return false;
    const int gb = __ldcg(&c->grid_b);
    if (gb == 0) return true;  // y == 0: nothing is ever added
    const int e = 1100 - gb;
    const double Y = __longlong_as_double((long long)__ldcg(&c->ymax));
    const double R = __longlong_as_double((long long)__ldcg(&c->rmax[it & 1]));
    const double X = __longlong_as_double((long long)__ldcg(&c->xmax[it & 1]));
    const double bound = Y + (double)__ldcg(&c->deg) * (X + 2.0 * R);
    if (e + 51 > 1023) return true;
    return bound < ldexp(1.0, e + 51);
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, v, o);
        v = t > v ? t : v;
    }
    return v;
}

// Residual phase of a problem whose incremental residual is exact: r_next
// already holds the new residual; copy the rows that changed into r, with
// their fingerprints, and return this warp's exact change of ||r||_0 and
// largest |r_i| (bits), both valid in every lane.
__device__ __forceinline__ long long residual_exact_tile(const ProblemDev &P, int tile, int lane,
                                                         unsigned long long &rmax) {
    const int i = tile * kTile + lane;
    long long delta = 0;
    unsigned long long mag = 0;
    if (i < P.m) {
        const double v = __ldcg(P.r_next + i), o = __ldcg(P.r + i);
        if (value_bits(v) != value_bits(o)) {
            P.r[i] = v;
            store_fp(P, i, v);
        }
        delta = (long long)(v != 0.0) - (long long)(o != 0.0);
        mag = value_bits(v) & 0x7fffffffffffffffull;
    }
    rmax = warp_max_u64(mag);
    return warp_sum_ll(delta);
}

// One row of the residual phase.  The touched flag, the row's slot record,
// y_i and the old r_i are independent loads issued together; only touched
// rows then gather their contributors' x_hat_j.
// One row tile of the residual phase.  Rows with more contributors than
// their slot record holds are appended to the CTA's overflow list (summed
// afterwards, one warp a row); when the list is full the warp sums them
// itself.
static __device__ __noinline__ long long residual_tile(const ProblemDev &P, int tile, int lane,
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
        store_fp(P, i, rn);
    }
    return warp_sum_ll(delta);
}

// A listed overflow row, by one warp; returns the row's change of ||r||_0.
static __device__ __noinline__ long long residual_overflow_row(const ProblemDev &P, int i, int lane) {
    const double s = warp_ordered_row_sum_flagged(P, i, lane);
    long long delta = 0;
    if (lane == 0) {
        const double rn = __dsub_rn(__ldg(P.y + i), s);
        const double ro = __ldcg(P.r + i);
        delta = (long long)(rn != 0.0) - (long long)(ro != 0.0);
        P.touched[i] = 0;
        P.r[i] = rn;
        store_fp(P, i, rn);
    }
    return delta;
}

// Init of one row: r <- y (both copies), fingerprint, empty record; and the
// row's part of ||y||_0 and of the certificate's constants (lowest set bit
// over the nonzero y_i, largest |y_i|, largest row degree).
struct InitStats {
    long long nz = 0;
    unsigned long long ymax = 0;
    int gridb = 0, deg = 0;
};

__device__ __forceinline__ void init_row(const ProblemDev &P, int i, InitStats &st) {
    const double v = __ldg(P.y + i);
    P.r[i] = v;
    P.r_next[i] = v;
    store_fp(P, i, v);
    P.touched[i] = 0;
    P.slots[(size_t)i * kSlotRec] = 0;
    const unsigned long long b = value_bits(v) & 0x7fffffffffffffffull;
    if (b) {
        ++st.nz;
        st.ymax = b > st.ymax ? b : st.ymax;
        st.gridb = max(st.gridb, 1100 - lowbit_exponent(b));
    }
    st.deg = max(st.deg, (int)(__ldg(P.csr_ptr + i + 1) - __ldg(P.csr_ptr + i)));
}

__device__ __forceinline__ void init_stats_begin(long long &s_sum, unsigned long long &s_umax,
                                                 int &s_gridb, int &s_deg) {
    if (threadIdx.x == 0) {
        s_sum = 0;
        s_umax = 0;
        s_gridb = 0;
        s_deg = 0;
    }
    __syncthreads();
}

// Warp, then CTA, then one set of global atomics per CTA and problem.
__device__ __forceinline__ void init_stats_end(const ProblemDev &P, const InitStats &st, int lane,
                                               long long &s_sum, unsigned long long &s_umax,
                                               int &s_gridb, int &s_deg) {
    const long long nz = warp_sum_ll(st.nz);
    const unsigned long long ym = warp_max_u64(st.ymax);
    const int gb = __reduce_max_sync(0xffffffffu, (unsigned)st.gridb);
    const int dg = __reduce_max_sync(0xffffffffu, (unsigned)st.deg);
    if (lane == 0) {
        if (nz) atomicAdd(reinterpret_cast<unsigned long long *>(&s_sum), (unsigned long long)nz);
        if (ym) atomicMax(&s_umax, ym);
        if (gb) atomicMax(&s_gridb, gb);
        if (dg) atomicMax(&s_deg, dg);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        DecodeCtrl *c = P.ctrl;
        if (s_sum) atomicAdd(reinterpret_cast<unsigned long long *>(&c->r0), (unsigned long long)s_sum);
        if (s_umax) {
            atomicMax(&c->ymax, s_umax);
            atomicMax(&c->rmax[0], s_umax);
        }
        if (s_gridb) atomicMax(&c->grid_b, s_gridb);
        if (s_deg) atomicMax(&c->deg, s_deg);
    }
}

template <int DMAX, int THREADS>
__global__ void __launch_bounds__(THREADS, 1) k_engine(const __grid_constant__ EngineArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int kWarps = THREADS / 32;
    __shared__ __align__(8) uint64_t s_bars[2 * kMaxStages + 1];
    __shared__ int s_qn;
    __shared__ unsigned long long s_acc;
    __shared__ long long s_sum;
    __shared__ unsigned long long s_xmax, s_umax;
    __shared__ int s_gridb, s_deg;
    __shared__ int s_ovf_n;
    __shared__ int s_ovf[kOvfCap];  // rows whose sum needs the whole CSR row
    __shared__ int s_rows_R, s_rows_E, s_rowmode;  // the iteration's row-driven phase
    __shared__ int s_wbuf[kUseWarpBuffer<THREADS, true>
                              ? (kWarps - 1) * kWbufPerWarp * kWbufEntry<DMAX> : 1];
    ScoreSmem S;
    S.fp = smem;
    S.stage = reinterpret_cast<char *>(smem + a.fp_cap);
    S.queue = reinterpret_cast<int32_t *>(S.stage + (size_t)a.stages * a.stage_bytes);
    int8_t *s_status = reinterpret_cast<int8_t *>(
        reinterpret_cast<char *>(S.queue) + ((a.queue_cap * (DMAX + 1) * 4 + 15) / 16) * 16);
    long long *s_pref = reinterpret_cast<long long *>(
        reinterpret_cast<char *>(s_status) + ((a.P + 15) / 16) * 16);  // a.P + 1 entries
    int *s_base = reinterpret_cast<int *>(s_pref + a.P + 1);          // a.P entries
    int8_t *s_rmode = reinterpret_cast<int8_t *>(s_base + a.P);        // a.P entries
    S.full = s_bars;
    S.empty = s_bars + kMaxStages;
    S.fp_bar = &s_bars[2 * kMaxStages];
    S.qn = &s_qn;
    S.acc = &s_acc;
    S.wbuf = s_wbuf;
    S.xmax = &s_xmax;
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
    // residual mode carried over from an earlier launch (0 for a fresh
    // problem); CTA 0 writes the flag only after the init barrier
    for (int p = threadIdx.x; p < a.P; p += THREADS)
        s_rmode[p] = (int8_t)(__ldcg(&problem(a, p).ctrl->ordered) ? 1 : 0);
    __syncthreads();

    // a lone problem: this CTA's column tiles are the same in every
    // iteration, so once the stop rule has let the problem run another
    // iteration, the fingerprint copy and the first CSC chunk of that score
    // phase are issued at once, ahead of the iteration's set-up (thread 0
    // keeps the record in shared memory)
    __shared__ Prefetch pf;
    constexpr int kPer = (kWarps - 1) * ((THREADS == 512) ? 2 : 1);  // tiles per chunk
    auto my_tiles = [&](int &t0, int &t1) {
        const long long tiles = (a.single.n + kTile - 1) / kTile;
        t0 = (int)(tiles * blockIdx.x / gridDim.x);
        t1 = (int)(tiles * (blockIdx.x + 1) / gridDim.x);
    };
    auto issue_ahead = [&](int g_next) {
        if (a.probs || threadIdx.x != 0 || g_next >= a.iter_budget || s_status[0] != kRunning)
            return;
        int t0, t1;
        my_tiles(t0, t1);
        if (t1 <= t0) return;
        if (a.single.flags & kPdUseFp) prefetch_fp(a.single, S, pf);
        // a row-driven iteration streams no CSC (its row list uses the ring)
        if (!row_driven_iter(a, a.single, s_base[0] + g_next, __ldcg(&a.single.ctrl->r0)))
            prefetch_chunks(a, a.single, t0, t1, kPer, S, chunk_seq, pf, ok);
    };
    if (threadIdx.x == 0) {
        pf.chunks = 0;
        pf.fp = false;
    }
    auto leave = [&]() {
        if (threadIdx.x == 0) drain_prefetch(a, S, chunk_seq, fp_seq, pf);
        fail_out(a);
    };

    // ---- init: x_hat <- 0, r <- y (Alg. 2, first line) --------------------
    if (!a.probs) {
        // one problem: grid-stride over its rows (x_hat <- 0 is stored by
        // the first score phase's stream, or below if the decode stops at
        // once; the in-slots flags are set when the ordered residual begins)
        const ProblemDev &P = a.single;
        const long long gtid = blockIdx.x * (long long)THREADS + threadIdx.x;
        const long long gstride = (long long)gridDim.x * THREADS;
        for (long long w = gtid; w < (P.n + 3) / 4; w += gstride) P.hits[w] = 0u;
        init_stats_begin(s_sum, s_umax, s_gridb, s_deg);
        InitStats st;
        for (long long i = gtid; i < P.m; i += gstride) init_row(P, (int)i, st);
        init_stats_end(P, st, lane, s_sum, s_umax, s_gridb, s_deg);
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
                            init_stats_begin(s_sum, s_umax, s_gridb, s_deg);
                            InitStats st;
                            for (int t = t0 + warp; t < t1; t += kWarps) {
                                const int i = t * kTile + lane;
                                if (i < P.m) init_row(P, i, st);
                            }
                            init_stats_end(P, st, lane, s_sum, s_umax, s_gridb, s_deg);
                        });
    }
    if (!grid_barrier(a, bar++)) {
        leave();
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
            P.ctrl->empty_run[0] = 0;
            P.ctrl->max_iter = a.max_iter;
            if (P.r0_hist) P.r0_hist[0] = r0;
        }
    }
    __syncthreads();
    if (!a.probs && s_status[0] != kRunning) {
        // a lone problem that stops before its first score phase (y == 0 or
        // max_iter == 0): x_hat <- 0 here
        const long long gtid = blockIdx.x * (long long)THREADS + threadIdx.x;
        for (long long j = gtid; j < a.single.n; j += (long long)gridDim.x * THREADS)
            a.single.x_hat[j] = 0.0;
    }
    issue_ahead(0);

    for (int g = 0; g < a.iter_budget; ++g) {
        int any = 0;
        for (int p = threadIdx.x; p < a.P; p += THREADS) any |= (s_status[p] == kRunning);
        if (!__syncthreads_or(any)) break;
        if (blockIdx.x == 0)
            for (int p = threadIdx.x; p < a.P; p += THREADS) problem(a, p).ctrl->acc[(g + 2) & 3] = 0;
        // residual mode of this iteration, per problem (the same decision in
        // every CTA: it reads maxima stored before the last grid barrier)
        for (int p = threadIdx.x; p < a.P; p += THREADS) {
            if (s_status[p] != kRunning || s_rmode[p] == 1) continue;
            const ProblemDev &P = problem(a, p);
            const int it = s_base[p] + g;
            if (s_rmode[p] == 2) {
                s_rmode[p] = 1;
            } else if (!exact_certified(P.ctrl, it, a.debug_flags)) {
                s_rmode[p] = 2;
                if (blockIdx.x == 0) P.ctrl->ordered = 1;
            } else if (blockIdx.x == 0) {
                P.ctrl->rmax[(it + 1) & 1] = 0;
                atomicMax(&P.ctrl->xmax[(it + 1) & 1], __ldcg(&P.ctrl->xmax[it & 1]));
            }
        }
        __syncthreads();

        // ---- score + apply ------------------------------------------------
        if (!a.probs) {
            int t0, t1;
            my_tiles(t0, t1);
            const int it = s_base[0] + g;
            const bool rows_mode = row_driven_iter(a, a.single, it, __ldcg(&a.single.ctrl->r0));
            if (threadIdx.x == 0) s_rowmode = rows_mode;
            if (rows_mode) {
                ok = score_rows<DMAX, THREADS>(a, a.single, t0, t1, g, it, s_rmode[0], S, fp_seq,
                                               ok, &pf, &s_rows_R, &s_rows_E);
                ++fp_seq;
            } else if (t1 > t0)
                score_segment<DMAX, THREADS>(a, a.single, t0, t1, g, it, s_rmode[0], S,
                                             chunk_seq, fp_seq, ok, &pf, /*zero_x=*/g == 0);
        } else {
            build_partition<THREADS>(a, s_status, s_pref, kPartScore);
            for_my_segments(a, s_status, s_pref, kPartScore,
                            [&](int p, const ProblemDev &P, int t0, int t1) {
                                if (!__syncthreads_and(ok)) return;
                                score_segment<DMAX, THREADS>(a, P, t0, t1, g, s_base[p] + g,
                                                             s_rmode[p], S, chunk_seq, fp_seq, ok);
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
            leave();
            return;
        }

        // ---- residual + ||r||_0 ---------------------------------------------
        auto residual_segment = [&](int p, const ProblemDev &P, int t0, int t1) {
            if (s_rmode[p] == 0) {
                // exact incremental residual: a streaming pass over the rows
                if (threadIdx.x == 0) {
                    s_sum = 0;
                    s_umax = 0;
                }
                __syncthreads();
                for (int t = t0 + warp; t < t1; t += kWarps) {
                    unsigned long long rmax;
                    const long long delta = residual_exact_tile(P, t, lane, rmax);
                    if (lane == 0) {
                        if (delta)
                            atomicAdd(reinterpret_cast<unsigned long long *>(&s_sum),
                                      (unsigned long long)delta);
                        if (rmax) atomicMax(&s_umax, rmax);
                    }
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    if (s_sum)
                        atomicAdd(reinterpret_cast<unsigned long long *>(&P.ctrl->r0),
                                  (unsigned long long)s_sum);
                    if (s_umax) atomicMax(&P.ctrl->rmax[(s_base[p] + g + 1) & 1], s_umax);
                }
                return;
            }
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
            residual_segment(0, a.single, (int)(tiles * blockIdx.x / gridDim.x),
                             (int)(tiles * (blockIdx.x + 1) / gridDim.x));
            __syncthreads();
            if (s_rowmode) row_hits_clear<THREADS>(a.single);
        } else {
            build_partition<THREADS>(a, s_status, s_pref, kPartRows);
            for_my_segments(a, s_status, s_pref, kPartRows,
                            [&](int p, const ProblemDev &P, int t0, int t1) {
                                residual_segment(p, P, t0, t1);
                            });
        }
        if (!grid_barrier(a, bar++)) {
            leave();
            return;
        }

        // ---- stop rule ("while not converged", three ways to stop) ----------
        // An iteration that accepts nothing stalls the decode; in the shifted
        // variant it only moves the candidate to the next position, and the
        // decode stalls when d iterations in a row accepted nothing (every
        // position tried on the same r).  The run length lives in a two-slot
        // ring by iteration parity: every CTA reads slot it & 1, CTA 0 writes
        // slot (it + 1) & 1, so the phase has no read-write race.
        for (int p = threadIdx.x; p < a.P; p += THREADS) {
            if (s_status[p] != kRunning) continue;
            const ProblemDev &P = problem(a, p);
            int st;
            const int it_now = s_base[p] + g;
            const bool empty = __ldcg(&P.ctrl->acc[g & 3]) == 0;
            const int run = empty ? __ldcg(&P.ctrl->empty_run[it_now & 1]) + 1 : 0;
            if (blockIdx.x == 0) P.ctrl->empty_run[(it_now + 1) & 1] = run;
            if (empty && run >= (a.shifted ? P.d : 1)) {
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
        issue_ahead(g + 1);
    }
    if (threadIdx.x == 0) drain_prefetch(a, S, chunk_seq, fp_seq, pf);
    // every problem has stopped: CTA 0 publishes the results on the device
    if (a.dev_out && blockIdx.x == 0) {
        for (int p = threadIdx.x; p < a.P; p += THREADS) {
            const ProblemDev &P = problem(a, p);
            ccs_result res;
            res.status = P.ctrl->status;
            res.iterations = P.ctrl->iteration;
            res.r0_final = __ldcg(&P.ctrl->r0);
            res.error = __ldcg(&a.sync->error) ? CCS_ETIMEOUT : CCS_OK;
            res.row_driven = P.ctrl->row_driven;
            res.row_entries = P.ctrl->row_entries;
            res.residual_form = P.ctrl->ordered ? CCS_RESIDUAL_ORDERED : CCS_RESIDUAL_EXACT;
            res.reserved = 0;
            a.dev_out[P.out_slot] = res;
        }
    }
}

typedef void (*engine_fn)(const EngineArgs);

// Instance getters, one per file ccs_engine_k<threads>_d<pair>.cu.
engine_fn engine_kernel_1024_d1(int dmax);  // DMAX 1 or 2
engine_fn engine_kernel_1024_d3(int dmax);  // DMAX 3 or 4
engine_fn engine_kernel_1024_d5(int dmax);  // DMAX 5 or 6
engine_fn engine_kernel_1024_d7(int dmax);  // DMAX 7 or 8
engine_fn engine_kernel_768_d1(int dmax);  // DMAX 1 or 2
engine_fn engine_kernel_768_d3(int dmax);  // DMAX 3 or 4
engine_fn engine_kernel_768_d5(int dmax);  // DMAX 5 or 6
engine_fn engine_kernel_768_d7(int dmax);  // DMAX 7 or 8
engine_fn engine_kernel_512_d1(int dmax);  // DMAX 1 or 2
engine_fn engine_kernel_512_d3(int dmax);  // DMAX 3 or 4
engine_fn engine_kernel_512_d5(int dmax);  // DMAX 5 or 6
engine_fn engine_kernel_512_d7(int dmax);  // DMAX 7 or 8
engine_fn engine_kernel_512_d9(int dmax);  // DMAX 9 or 10
engine_fn engine_kernel_512_d11(int dmax);  // DMAX 11 or 12
engine_fn engine_kernel_512_d13(int dmax);  // DMAX 13 or 14
engine_fn engine_kernel_512_d15(int dmax);  // DMAX 15 or 16

}  // namespace ccs

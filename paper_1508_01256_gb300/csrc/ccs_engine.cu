// ccs_engine.cu -- Parallel-l0 (Alg. 2) in one persistent cooperative launch.
//
// One launch runs every iteration of one or many independent problems.  The
// grid is one CTA per SM (co-resident by cooperative launch); the phases of an
// iteration are separated by grid barriers:
//
//   init      x_hat <- 0, r <- y, fingerprints of r, ||y||_0
//   score     every column of every running problem: exact score (Eq. (15)
//             or Alg. 8) and, if accepted, x_hat_j += omega_j (apply).  The
//             problem's 8-bit residual fingerprints sit in shared memory when
//             they fit, so most columns are rejected from on-chip data alone
//             (a fingerprint count bounds every value's count); only the
//             columns that may reach alpha gather their d binary64 values.
//   residual  every touched row: r_i = y_i - ordered sum of its nonzero
//             x_hat_j, new fingerprint, exact change of ||r||_0
//   stop      every CTA applies the stop rule to every problem from the same
//             counters, so all CTAs agree without another barrier
//
// Work unit: a tile of 32 columns (score) or 32 rows (residual), one warp.
// A CTA owns a contiguous range of tiles, so it loads one problem's
// fingerprints once per phase.  Every barrier wait is bounded by the
// watchdog: on time-out the CTA records kErrWatchdog and returns, and the
// host reports CCS_ETIMEOUT.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "ccs_device.cuh"

namespace ccs {

constexpr int kTile = 32;
constexpr int kMaxBlocks = 1024;
constexpr int kMaxStampIters = 1024;
constexpr int kFlagSkipArrive = 1;  // test hook: CTA 0 never arrives at barrier 1

struct Segment {
    int prob, lo, hi, pad;  // tiles [lo, hi) of problem `prob`
};

struct EngineArgs {
    ProblemDev single;          // used when probs == nullptr (one problem)
    const ProblemDev *probs;    // P descriptors in device memory
    int P;
    int alpha, mode, max_iter;
    int fp_cap;                 // bytes of the shared fingerprint buffer
    int stride;                 // ints per column in a warp's index stage (odd)
    const int *score_ptr;       // G+1 offsets into score_segs (batch only)
    const Segment *score_segs;
    const int *res_ptr;
    const Segment *res_segs;
    unsigned *arrive;           // monotonic barrier counter
    int *error;                 // ErrorBits for the whole launch
    unsigned long long *stamps; // globaltimer after each barrier (or null)
    long long watchdog_ns;
    int debug_flags;
};

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

// Grid barrier number `index` (0-based).  Returns false if the wait ran past
// the watchdog (or another CTA already gave up).
__device__ bool grid_barrier(const EngineArgs &a, unsigned index, bool arrive = true) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (arrive) {
            __threadfence();
            atomicAdd(a.arrive, 1u);
        }
        const unsigned target = (index + 1u) * gridDim.x;
        const unsigned long long t0 = globaltimer();
        while (ld_acquire(a.arrive) < target) {
            if (*reinterpret_cast<volatile int *>(a.error) != 0 ||
                globaltimer() - t0 > (unsigned long long)a.watchdog_ns) {
                atomicOr(a.error, kErrWatchdog);
                ok = 0;
                break;
            }
            __nanosleep(64);
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

// Stage the d row indices of a tile's columns in shared memory (stride
// `stride` per column, odd, so that lane-strided reads hit distinct banks).
__device__ __forceinline__ void stage_tile(const ProblemDev &P, int base, int cols, int stride,
                                           int32_t *stage, int lane) {
    const int d = P.d;
    const int32_t *src = P.csc_rows + (size_t)base * d;
    const int total = cols * d;
    if (((reinterpret_cast<uintptr_t>(src) & 15u) == 0) && (total & 3) == 0) {
        const int4 *src4 = reinterpret_cast<const int4 *>(src);
        for (int q = lane; q < (total >> 2); q += 32) {
            const int4 v = __ldg(src4 + q);
            int e = q << 2;
            int col = e / d, t = e - col * d;
            const int vals[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                stage[col * stride + t] = vals[u];
                if (++t == d) {
                    t = 0;
                    ++col;
                }
            }
        }
    } else {
        for (int e = lane; e < total; e += 32) {
            const int col = e / d;
            stage[col * stride + (e - col * d)] = __ldg(src + e);
        }
    }
}

template <int DMAX>
__device__ __forceinline__ bool score_tile(const EngineArgs &a, const ProblemDev &P, int tile,
                                           const uint8_t *s_fp, int32_t *stage, int lane) {
    const int base = tile * kTile;
    const int cols = min(kTile, P.n - base);
    stage_tile(P, base, cols, a.stride, stage, lane);
    __syncwarp();
    bool acc = false;
    if (lane < cols) {
        const int32_t *rows = stage + lane * a.stride;
        const bool cand = s_fp ? may_accept<DMAX>(s_fp, rows, P.d, a.alpha, a.mode) : true;
        if (cand) {
            unsigned long long omega;
            acc = exact_score<DMAX>(rows, P.d, P.r, a.alpha, a.mode, &omega);
            if (acc) apply_pair(P, base + lane, rows, P.d, omega);
        }
    }
    __syncwarp();
    return acc;
}

__device__ __forceinline__ long long residual_tile(const ProblemDev &P, int tile, int lane) {
    const int i = tile * kTile + lane;
    long long delta = 0;
    if (i < P.m && __ldcg(P.touched + i)) {
        P.touched[i] = 0;
        const double rn = row_residual(P, i);
        const double ro = __ldcg(P.r + i);
        delta = (long long)(rn != 0.0) - (long long)(ro != 0.0);
        P.r[i] = rn;
        P.fp[i] = fingerprint(rn);
    }
    return warp_sum_ll(delta);
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
        L.segs = nullptr;  // use `one`
        L.count = 1;
    } else {
        const int *ptr = score ? a.score_ptr : a.res_ptr;
        L.segs = (score ? a.score_segs : a.res_segs) + ptr[blockIdx.x];
        L.count = ptr[blockIdx.x + 1] - ptr[blockIdx.x];
        L.one = Segment{0, 0, 0, 0};
    }
    return L;
}

template <int DMAX, int THREADS>
__global__ void __launch_bounds__(THREADS, 1) k_engine(const __grid_constant__ EngineArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint8_t *s_fp = smem;
    int32_t *s_stage = reinterpret_cast<int32_t *>(smem + a.fp_cap);
    constexpr int kWarps = THREADS / 32;
    int8_t *s_status = reinterpret_cast<int8_t *>(s_stage + kWarps * kTile * a.stride);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int32_t *stage = s_stage + warp * kTile * a.stride;
    unsigned bar = 0;

    // ---- init: x_hat <- 0, r <- y (Alg. 2, first line) --------------------
    const long long gtid = blockIdx.x * (long long)THREADS + threadIdx.x;
    const long long gstride = (long long)gridDim.x * THREADS;
    for (int p = 0; p < a.P; ++p) {
        const ProblemDev &P = problem(a, p);
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
            P.slot_cnt[i] = 0;
            nz += (v != 0.0);
        }
        nz = warp_sum_ll(nz);
        if (lane == 0 && nz)
            atomicAdd(reinterpret_cast<unsigned long long *>(&P.ctrl->r0), (unsigned long long)nz);
    }
    if (!grid_barrier(a, bar++)) return;
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
                if (s_status[sg.prob] != kRunning) continue;
                const ProblemDev &P = problem(a, sg.prob);
                const bool use_fp = P.pad != 0;
                if (use_fp) {
                    __syncthreads();
                    const int4 *src = reinterpret_cast<const int4 *>(P.fp);
                    int4 *dst = reinterpret_cast<int4 *>(s_fp);
                    const int n16 = (P.m + 15) >> 4;
                    for (int q = threadIdx.x; q < n16; q += THREADS) dst[q] = __ldcg(src + q);
                    __syncthreads();
                }
                unsigned long long *acc_slot = &P.ctrl->acc[g & 3];
                for (int t = sg.lo + warp; t < sg.hi; t += kWarps) {
                    const bool acc = score_tile<DMAX>(a, P, t, use_fp ? s_fp : nullptr, stage, lane);
                    const unsigned bal = __ballot_sync(0xffffffffu, acc);
                    if (lane == 0 && bal) atomicAdd(acc_slot, (unsigned long long)__popc(bal));
                }
            }
        }
        const bool skip = (a.debug_flags & kFlagSkipArrive) && blockIdx.x == 0 && g == 0;
        if (!grid_barrier(a, bar++, !skip) || skip) return;

        // ---- residual + ||r||_0 ---------------------------------------------
        {
            const SegList L = my_segments(a, false);
            for (int s = 0; s < L.count; ++s) {
                const Segment sg = L.segs ? L.segs[s] : L.one;
                if (s_status[sg.prob] != kRunning) continue;
                const ProblemDev &P = problem(a, sg.prob);
                for (int t = sg.lo + warp; t < sg.hi; t += kWarps) {
                    const long long delta = residual_tile(P, t, lane);
                    if (lane == 0 && delta)
                        atomicAdd(reinterpret_cast<unsigned long long *>(&P.ctrl->r0),
                                  (unsigned long long)delta);
                }
            }
        }
        if (!grid_barrier(a, bar++)) return;

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
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

constexpr int kSmemLimit = 227 * 1024;

static int stride_for(int dmax) { return dmax | 1; }
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

// Fixed engine bytes of the workspace for P problems.
size_t engine_ws_bytes(int P) {
    size_t b = 0;
    b += align_up(sizeof(unsigned) * 2, 256);                           // arrive, error
    b += align_up(sizeof(unsigned long long) * (3 * kMaxStampIters + 2), 256);  // stamps
    if (P > 1) {
        b += align_up(sizeof(ProblemDev) * (size_t)P, 256);
        b += 2 * align_up(sizeof(int) * (kMaxBlocks + 1), 256);
        b += 2 * align_up(sizeof(Segment) * (size_t)(kMaxBlocks + P), 256);
    }
    return b;
}

struct DeviceInfo {
    int sms = 0;
    int coop = 0;
};

static DeviceInfo device_info() {
    static std::mutex mu;
    static int cached_dev = -1;
    static DeviceInfo cached;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (dev != cached_dev) {
        cudaDeviceGetAttribute(&cached.sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&cached.coop, cudaDevAttrCooperativeLaunch, dev);
        cached_dev = dev;
    }
    return cached;
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

// Launch the engine on P problems whose workspaces are already carved out in
// `pds`; `eng` points at the engine area.  Fills out[0..P).
int engine_run(std::vector<ProblemDev> &pds, const ccs_params &prm, ccs_result *out, char *eng,
               cudaStream_t s) {
    const int P = (int)pds.size();
    int dmax = 1;
    for (auto &pd : pds) dmax = std::max(dmax, pd.d);
    engine_fn fn = engine_kernel(dmax);
    const int threads = threads_for(dmax);
    const int stride = stride_for(dmax);
    const size_t stage_bytes = (size_t)(threads / 32) * kTile * stride * 4;
    const size_t status_bytes = align_up((size_t)P, 16);
    if (stage_bytes + status_bytes + 1024 > (size_t)kSmemLimit) {
        set_last_error("too many problems in one launch (%d)", P);
        return CCS_EINVAL;
    }
    const size_t fp_budget = (size_t)kSmemLimit - stage_bytes - status_bytes - 1024;
    size_t fp_cap = 0;
    for (auto &pd : pds) {
        const size_t need = align_up((size_t)pd.m, 16);
        pd.pad = need <= fp_budget ? 1 : 0;
        if (pd.pad) fp_cap = std::max(fp_cap, need);
    }
    const size_t smem = fp_cap + stage_bytes + status_bytes;

    const DeviceInfo di = device_info();
    if (!di.coop) {
        set_last_error("device does not support cooperative launches");
        return CCS_ECUDA;
    }
    CCS_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    CCS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem));
    if (per_sm < 1) {
        set_last_error("engine kernel does not fit on an SM (smem %zu)", smem);
        return CCS_ECUDA;
    }
    const int G = std::min(kMaxBlocks, di.sms * std::min(per_sm, 1));

    EngineArgs a;
    std::memset(&a, 0, sizeof(a));
    a.P = P;
    a.alpha = prm.alpha;
    a.mode = prm.score_mode;
    a.max_iter = prm.max_iter;
    a.fp_cap = (int)fp_cap;
    a.stride = stride;
    a.watchdog_ns = (long long)(prm.watchdog_ms > 0 ? prm.watchdog_ms : 2000) * 1000000ll;
    a.debug_flags = prm.debug_flags;

    char *e = eng;
    a.arrive = reinterpret_cast<unsigned *>(e);
    a.error = reinterpret_cast<int *>(e + sizeof(unsigned));
    e += align_up(sizeof(unsigned) * 2, 256);
    unsigned long long *stamps = reinterpret_cast<unsigned long long *>(e);
    e += align_up(sizeof(unsigned long long) * (3 * kMaxStampIters + 2), 256);
    a.stamps = profiling() ? stamps : nullptr;

    // control blocks and barrier state start at zero
    for (auto &pd : pds) CCS_CUDA_TRY(cudaMemsetAsync(pd.ctrl, 0, sizeof(DecodeCtrl), s));
    CCS_CUDA_TRY(cudaMemsetAsync(eng, 0, sizeof(unsigned) * 2, s));

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

    // results
    std::vector<DecodeCtrl> hc(P);
    for (int p = 0; p < P; ++p)
        CCS_CUDA_TRY(cudaMemcpyAsync(&hc[p], pds[p].ctrl, sizeof(DecodeCtrl),
                                     cudaMemcpyDeviceToHost, s));
    int herr = 0;
    CCS_CUDA_TRY(cudaMemcpyAsync(&herr, a.error, sizeof(int), cudaMemcpyDeviceToHost, s));
    std::vector<unsigned long long> hst;
    if (a.stamps) {
        hst.resize(3 * kMaxStampIters + 2);
        CCS_CUDA_TRY(cudaMemcpyAsync(hst.data(), stamps, sizeof(unsigned long long) * hst.size(),
                                     cudaMemcpyDeviceToHost, s));
    }
    CCS_CUDA_TRY(cudaStreamSynchronize(s));
    int max_it = 0;
    for (int p = 0; p < P; ++p) {
        out[p].status = hc[p].status;
        out[p].iterations = hc[p].iteration;
        out[p].r0_final = hc[p].r0;
        out[p].error = herr ? CCS_ETIMEOUT : CCS_OK;
        out[p].reserved = 0;
        max_it = std::max(max_it, hc[p].iteration);
    }
    if (a.stamps && !herr) {
        // barrier 0 ends init; iteration g: score ends at 1+2g, residual at 2+2g
        for (int g = 0; g < max_it && 2 + 2 * g < (int)hst.size(); ++g) {
            const unsigned long long t0 = hst[2 * g], t1 = hst[1 + 2 * g], t2 = hst[2 + 2 * g];
            if (t1 >= t0 && t2 >= t1 && t0) {
                prof_add(CCS_K_SCORE, (t1 - t0) * 1e-6);
                prof_add(CCS_K_RESIDUAL, (t2 - t1) * 1e-6);
            }
        }
    }
    if (herr) {
        set_last_error("a grid barrier wait exceeded the watchdog (%d ms)",
                       prm.watchdog_ms > 0 ? prm.watchdog_ms : 2000);
        return CCS_ETIMEOUT;
    }
    return CCS_OK;
}

}  // namespace ccs

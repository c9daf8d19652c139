// ccs_engine.cu -- host side of the persistent engine: launch planning
// (kernel instance, shared-memory plan, grid), one-shot and captured
// launches, and resume-mode launches for the server.  The kernel itself is
// in ccs_engine_kernel.cuh.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <tuple>
#include <vector>

#include "ccs_engine_kernel.cuh"

namespace ccs {

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

// Launch shape (ccs_params.schedule): bits 0-1 the thread shape
// (threads per CTA, tiles per consumer warp and chunk),
//   1: 1024 threads, 1 tile  (d <= 8: at most 64 registers a thread)
//   2:  512 threads, 2 tiles (any d: up to 128 registers a thread)
//   3:  768 threads, 1 tile  (d <= 8: up to 85 registers a thread)
// (0: the library's choice); bits 2-4 a cap on the CSC stages (0: as many
// as shared memory holds, else 2..6); bits 5-6 a cap on the candidate
// queue (0: as long as shared memory allows, 1: 256 entries, 2: 1024).
static int schedule_for(int dmax, int requested) {
    requested &= 3;
    if (requested == 2 || dmax > 8) return 2;
    if (requested == 3) return 3;
    return 1;  // measured fastest for d <= 8
}
static int stage_cap_of(int schedule) { return (schedule >> 2) & 7; }
static int queue_cap_of(int schedule) {
    const int q = (schedule >> 5) & 3;
    return q == 1 ? 256 : (q == 2 ? 1024 : kQueueCap);
}

// Launch shapes picked by ccs_autotune, by device, largest d of a launch and
// whether all its problems keep fingerprints in shared memory (0: none).
static std::mutex g_tune_mu;
static int g_tuned[64][kMaxD + 1][2];

void tuned_schedule_set(int dev, int dmax, bool fits, int schedule) {
    if (dev < 0 || dev >= 64 || dmax < 1 || dmax > kMaxD) return;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[dev][dmax][fits ? 1 : 0] = schedule;
}

static int tuned_schedule_get(int dev, int dmax, bool fits) {
    if (dev < 0 || dev >= 64 || dmax < 1 || dmax > kMaxD) return 0;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_tuned[dev][dmax][fits ? 1 : 0];
}

void tuned_schedule_reset() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    std::memset(g_tuned, 0, sizeof(g_tuned));
}

static engine_fn engine_kernel(int dmax, int schedule) {
    const int threads = schedule == 1 ? 1024 : (schedule == 3 ? 768 : 512);
    if (dmax < 1 || dmax > (threads == 512 ? 16 : 8)) return nullptr;
    const int lo = (dmax - 1) / 2 * 2 + 1;  // first DMAX of the instance pair
    switch (threads * 100 + lo) {
        case 102401: return engine_kernel_1024_d1(dmax);
        case 102403: return engine_kernel_1024_d3(dmax);
        case 102405: return engine_kernel_1024_d5(dmax);
        case 102407: return engine_kernel_1024_d7(dmax);
        case 76801: return engine_kernel_768_d1(dmax);
        case 76803: return engine_kernel_768_d3(dmax);
        case 76805: return engine_kernel_768_d5(dmax);
        case 76807: return engine_kernel_768_d7(dmax);
        case 51201: return engine_kernel_512_d1(dmax);
        case 51203: return engine_kernel_512_d3(dmax);
        case 51205: return engine_kernel_512_d5(dmax);
        case 51207: return engine_kernel_512_d7(dmax);
        case 51209: return engine_kernel_512_d9(dmax);
        case 51211: return engine_kernel_512_d11(dmax);
        case 51213: return engine_kernel_512_d13(dmax);
        case 51215: return engine_kernel_512_d15(dmax);
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
    int requested = prm.schedule;
    if ((requested & 3) == 0 && (requested >> 2) == 0) {
        // a shape picked by ccs_autotune for this class of launch, if any
        int dev = 0;
        CCS_CUDA_TRY(cudaGetDevice(&dev));
        bool fits_all = true;
        for (int p = 0; p < P && fits_all; ++p) fits_all = engine_fp_fits(pds[p], prm);
        const int t = tuned_schedule_get(dev, dmax, fits_all);
        if (t) requested = t;
    }
    int sched = schedule_for(dmax, requested);
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
                                sizeof(int) * (size_t)P + (size_t)P;  // + residual modes
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
        const size_t need = align_up((size_t)pd.m * (fp16_for(pd.m) ? 2 : 1), 16);
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
    int stages = (int)std::min<size_t>(kMaxStages, (smem_limit - fixed - fp_cap) / stage_bytes);
    if (stage_cap_of(requested) >= 2) stages = std::min(stages, stage_cap_of(requested));
    const size_t left = smem_limit - fp_cap - (size_t)stages * stage_bytes - status_bytes - 256;
    const int queue_cap = (int)std::min<size_t>(
        std::min(kQueueCap, queue_cap_of(requested)), (left - 16) / entry);
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
    a.shifted = prm.shifted;
    a.iter_budget = 0x7fffffff;
}


bool engine_fp_fits(const ProblemDev &pd, const ccs_params &prm) {
    // the fingerprint part of plan_launch for one problem, without the
    // occupancy query (called once per problem of a batch)
    const int sched = schedule_for(pd.d, prm.schedule);
    engine_fn fn = engine_kernel(pd.d, sched);
    int dev = 0;
    if (!fn || cudaGetDevice(&dev) != cudaSuccess) return false;
    const size_t smem_limit = max_dynamic_smem(dev, fn);
    const int threads = sched == 1 ? 1024 : (sched == 3 ? 768 : 512);
    const int tpw = sched == 2 ? 2 : 1;
    const size_t stage_bytes = align_up((size_t)(threads / 32 - 1) * tpw * kTile * pd.d * 4, 128);
    const size_t status_bytes = 16 + sizeof(long long) * 2 + sizeof(int) + 1;
    const size_t fixed = status_bytes + 256 + kMinQueue * (size_t)(pd.d + 1) * 4;
    if (smem_limit < fixed + 2 * stage_bytes) return false;
    const size_t need = align_up((size_t)pd.m * (fp16_for(pd.m) ? 2 : 1), 16);
    return need <= smem_limit - fixed - 2 * stage_bytes;
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
        out[p].row_driven = hc.row_driven;
        out[p].row_entries = hc.row_entries;
        out[p].residual_form = hc.ordered ? CCS_RESIDUAL_ORDERED : CCS_RESIDUAL_EXACT;
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

// Enqueue one resume-mode launch (no host wait).  Results go to dev_out,
// each at its problem's out_slot, or to the header's result area.
static int engine_resume_launch(ProblemDev *pds, int P, const ccs_params &prm, int iter_budget,
                                char *hdr, cudaStream_t s, ccs_result *dev_out) {
    LaunchPlan L;
    int rc = plan_launch(pds, P, prm, L);
    if (rc) return rc;
    EngineArgs a;
    fill_args(a, L, P, prm);
    a.resume = 1;
    a.iter_budget = iter_budget > 0 ? iter_budget : 1;
    a.sync = reinterpret_cast<EngineSync *>(hdr);
    a.dev_out = dev_out ? dev_out : reinterpret_cast<ccs_result *>(hdr + sizeof(EngineSync));
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
    return CCS_OK;
}

// A batch whose launch classes (groups) would each end in their own long
// tail of problems that iterate to max_iter: every group first runs alone,
// freshly initialised, for at most group_iters iterations; then one launch
// over every problem of the batch resumes the ones still running, so the
// groups' tails share iterations.  pds: the groups' descriptors back to back
// (their out_slot the caller's index, their control blocks distinct, in
// `ctrl_hdr`, `count` of them); rhdr: engine_resume_header_bytes(count)
// bytes.  Results: dev_out (each at out_slot), or host_out[out_slot].
int engine_run_phased(ProblemDev *pds, const int *sizes, int groups, int count,
                      const ccs_params &prm, int group_iters, char *ctrl_hdr, char *rhdr,
                      cudaStream_t s, ccs_result *dev_out, ccs_result *host_out) {
    CCS_CUDA_TRY(cudaMemsetAsync(ctrl_hdr, 0, sync_bytes(count), s));
    for (int t = 0; t < count; ++t) pds[t].flags |= kPdFresh;
    for (int g = 0, first = 0; g < groups; first += sizes[g], ++g) {
        int rc = engine_resume_launch(pds + first, sizes[g], prm, group_iters, rhdr, s, nullptr);
        if (rc) return rc;
    }
    for (int t = 0; t < count; ++t) pds[t].flags &= ~kPdFresh;
    int rc = engine_resume_launch(pds, count, prm, 0x7fffffff, rhdr, s, dev_out);
    if (rc || dev_out) return rc;
    const size_t bytes = sizeof(EngineSync) + sizeof(ccs_result) * (size_t)count;
    std::vector<char> h(bytes);
    CCS_CUDA_TRY(cudaMemcpyAsync(h.data(), rhdr, bytes, cudaMemcpyDeviceToHost, s));
    CCS_CUDA_TRY(cudaStreamSynchronize(s));
    EngineSync hs;
    std::memcpy(&hs, h.data(), sizeof(hs));
    std::memcpy(host_out, h.data() + sizeof(EngineSync), sizeof(ccs_result) * (size_t)count);
    if (hs.error) {
        for (int t = 0; t < count; ++t) host_out[t].error = CCS_ETIMEOUT;
        set_last_error("a bounded device wait exceeded the watchdog");
        return CCS_ETIMEOUT;
    }
    return CCS_OK;
}

// engine_run_phased captured in a CUDA graph: the control blocks' reset,
// each group's capped launch and the final launch over the whole batch.
// The descriptors are uploaded now, outside the capture: the groups' (fresh)
// to the launch header's descriptor area, the final launch's to the resume
// header's.  Results of the final launch go to dev_out.
int engine_capture_phased(ProblemDev *pds, const int *sizes, int groups, int count,
                          const ccs_params &prm, int group_iters, char *ctrl_hdr, char *rhdr,
                          ccs_result *dev_out, cudaGraphExec_t *exec) {
    std::vector<ProblemDev> fresh(pds, pds + count), resumed(pds, pds + count);
    for (int t = 0; t < count; ++t) {
        fresh[t].flags |= kPdFresh;
        resumed[t].flags &= ~kPdFresh;
    }
    ProblemDev *d_fresh =
        reinterpret_cast<ProblemDev *>(ctrl_hdr + sync_bytes(count) + stamps_bytes());
    ProblemDev *d_resumed =
        reinterpret_cast<ProblemDev *>(rhdr + resume_results_bytes(count) + stamps_bytes());
    std::vector<EngineArgs> args(groups + 1);
    std::vector<LaunchPlan> plans(groups + 1);
    for (int g = 0, first = 0; g <= groups; ++g) {
        const bool last = g == groups;
        const int P = last ? count : sizes[g];
        ProblemDev *host = last ? resumed.data() : fresh.data() + first;
        int rc = plan_launch(host, P, prm, plans[g]);
        if (rc) return rc;
        EngineArgs &a = args[g];
        fill_args(a, plans[g], P, prm);
        a.resume = 1;
        a.iter_budget = last ? 0x7fffffff : (group_iters > 0 ? group_iters : 1);
        a.sync = reinterpret_cast<EngineSync *>(rhdr);
        a.dev_out = last ? dev_out : reinterpret_cast<ccs_result *>(rhdr + sizeof(EngineSync));
        a.stamps = nullptr;
        a.probs = last ? d_resumed : d_fresh + first;
        if (!last) first += sizes[g];
    }
    // upload with the flags plan_launch set
    CCS_CUDA_TRY(cudaMemcpy(d_fresh, fresh.data(), sizeof(ProblemDev) * count,
                            cudaMemcpyHostToDevice));
    CCS_CUDA_TRY(cudaMemcpy(d_resumed, resumed.data(), sizeof(ProblemDev) * count,
                            cudaMemcpyHostToDevice));
    cudaStream_t cs;
    CCS_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e1 = cudaMemsetAsync(ctrl_hdr, 0, sync_bytes(count), cs);
        for (int g = 0; g <= groups && e1 == cudaSuccess; ++g) {
            const LaunchPlan &L = plans[g];
            void *kargs[] = {&args[g]};
            e1 = cudaMemsetAsync(rhdr, 0, sizeof(EngineSync), cs);
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
    if (e != cudaSuccess) return cuda_fail(e, "capturing the phased batch");
    return CCS_OK;
}

int engine_resume(ProblemDev *pds, int P, const ccs_params &prm, int iter_budget, ccs_result *out,
                  char *hdr, cudaStream_t s) {
    int rc = engine_resume_launch(pds, P, prm, iter_budget, hdr, s, nullptr);
    if (rc) return rc;
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

extern "C" CCS_API void ccs_autotune_reset(void) { ccs::tuned_schedule_reset(); }

namespace ccs {

// The tuned table on disk is keyed by GPU: its name, SM count and compute
// capability (one key per model, so a file written on one GB300 serves
// every GB300).
static bool gpu_key(int dev, char *out, size_t cap) {
    cudaDeviceProp pr;
    if (cudaGetDeviceProperties(&pr, dev) != cudaSuccess) return false;
    size_t k = 0;
    for (const char *c = pr.name; *c && k + 1 < cap; ++c) out[k++] = (*c == ' ') ? '_' : *c;
    out[k] = 0;
    std::snprintf(out + k, cap - k, "/sm%d/cc%d.%d", pr.multiProcessorCount, pr.major, pr.minor);
    return true;
}

}  // namespace ccs

extern "C" CCS_API int ccs_autotune_get(int32_t dmax, int32_t fits, int32_t *schedule) {
    if (!schedule || dmax < 1 || dmax > ccs::kMaxD) {
        ccs::set_last_error("ccs_autotune_get: bad arguments");
        return CCS_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ccs::cuda_fail(cudaGetLastError(), "cudaGetDevice");
    *schedule = ccs::tuned_schedule_get(dev, dmax, fits != 0);
    return CCS_OK;
}

extern "C" CCS_API int ccs_autotune_save(const char *path) {
    if (!path) return CCS_EINVAL;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) count = 0;
    FILE *f = std::fopen(path, "w");
    if (!f) {
        ccs::set_last_error("ccs_autotune_save: cannot write %s", path);
        return CCS_EINVAL;
    }
    std::fprintf(f, "# ccs launch shapes: gpu dmax fits schedule\n");
    for (int dev = 0; dev < count && dev < 64; ++dev) {
        char key[256];
        if (!ccs::gpu_key(dev, key, sizeof key)) continue;
        for (int dm = 1; dm <= ccs::kMaxD; ++dm)
            for (int fits = 0; fits < 2; ++fits) {
                const int sc = ccs::tuned_schedule_get(dev, dm, fits != 0);
                if (sc) std::fprintf(f, "%s %d %d %d\n", key, dm, fits, sc);
            }
    }
    const int bad = std::fclose(f);
    return bad ? CCS_EINVAL : CCS_OK;
}

extern "C" CCS_API int ccs_autotune_load(const char *path) {
    if (!path) return CCS_EINVAL;
    FILE *f = std::fopen(path, "r");
    if (!f) {
        ccs::set_last_error("ccs_autotune_load: cannot read %s", path);
        return CCS_EINVAL;
    }
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) count = 0;
    char line[512];
    while (std::fgets(line, sizeof line, f)) {
        char key[256];
        int dm = 0, fits = 0, sc = 0;
        if (line[0] == '#' || std::sscanf(line, "%255s %d %d %d", key, &dm, &fits, &sc) != 4)
            continue;
        if (dm < 1 || dm > ccs::kMaxD || (fits != 0 && fits != 1) || sc <= 0 || sc >= 128)
            continue;
        for (int dev = 0; dev < count && dev < 64; ++dev) {
            char mine[256];
            if (ccs::gpu_key(dev, mine, sizeof mine) && std::strcmp(mine, key) == 0)
                ccs::tuned_schedule_set(dev, dm, fits != 0, sc);
        }
    }
    std::fclose(f);
    return CCS_OK;
}

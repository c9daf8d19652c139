// ccs_batch.cu -- many independent decodes in one persistent launch.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "ccs_checks.cuh"
#include "ccs_internal.cuh"

namespace ccs {

// Iterations each launch group of a batch runs alone before the launch that
// merges the groups' tails (most converging problems finish within it).
constexpr int kGroupIters = 16;

static size_t batch_ws(const ccs_problem *probs, int32_t count) {
    size_t total = 0;
    for (int32_t q = 0; q < count; ++q) {
        if (check_sizes(probs[q].n, probs[q].m, probs[q].d) != CCS_OK) return 0;
        total += decode_ws_layout(probs[q].n, probs[q].m, nullptr, nullptr);
    }
    // launch header, then the header of the resume-mode launches that merge
    // the groups' tails, then each problem's arrays
    return engine_header_bytes(count) + engine_resume_header_bytes(count) + total;
}

// Time every launch shape for each launch group and record the fastest for
// the group's class.  The shapes: the thread shapes the kernel instances
// offer (d <= 8: 1024, 768 and 512 threads; d > 8: 512 only), each with
// the CSC ring as deep as shared memory allows or capped at 2 or 3 stages,
// and the candidate queue as long as shared memory allows or capped at 256
// entries (a shorter ring or queue leaves shared memory idle, but a deeper
// one delays the first chunk's consumers and the queue's scoring round).
// Each candidate decodes the group twice; the second run is timed.
// tuned[g] receives group g's choice (0..3 more entries are set to 0).
static int autotune_groups(std::vector<ProblemDev> &sub, const int *sizes, int groups,
                           const ccs_params &p, char *hdr, cudaStream_t s, int32_t *tuned) {
    int dev = 0;
    CCS_CUDA_TRY(cudaGetDevice(&dev));
    cudaEvent_t e0, e1;
    CCS_CUDA_TRY(cudaEventCreate(&e0));
    CCS_CUDA_TRY(cudaEventCreate(&e1));
    std::vector<ccs_result> part(sub.size());
    int rc = CCS_OK;
    for (int g = 0; g < 4; ++g) tuned[g] = 0;
    for (int g = 0, first = 0; g < groups && rc == CCS_OK; first += sizes[g], ++g) {
        int dmax = 1;
        bool fits = true;
        for (int u = 0; u < sizes[g]; ++u) {
            dmax = std::max(dmax, sub[first + u].d);
            fits = fits && engine_fp_fits(sub[first + u], p);
        }
        const int shapes_small[3] = {1, 3, 2}, shapes_large[1] = {2};
        const int *shapes = dmax <= 8 ? shapes_small : shapes_large;
        const int nshape = dmax <= 8 ? 3 : 1;
        const int stage_caps[3] = {0, 2, 3}, queue_codes[2] = {0, 1};
        int cands[18];
        int ncand = 0;
        for (int t = 0; t < nshape; ++t)
            for (int sc : stage_caps)
                for (int qc : queue_codes) cands[ncand++] = shapes[t] | (sc << 2) | (qc << 5);
        int best = 0;
        float best_ms = 0.0f;
        for (int c = 0; c < ncand && rc == CCS_OK; ++c) {
            ccs_params q = p;
            q.schedule = cands[c];
            float ms = 0.0f;
            for (int rep = 0; rep < 2 && rc == CCS_OK; ++rep) {
                if (cudaEventRecord(e0, s) != cudaSuccess) rc = CCS_ECUDA;
                if (rc == CCS_OK)
                    rc = engine_run(sub.data() + first, sizes[g], q, part.data() + first, hdr, s);
                if (rc == CCS_OK && (cudaEventRecord(e1, s) != cudaSuccess ||
                                     cudaEventSynchronize(e1) != cudaSuccess ||
                                     cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                    rc = CCS_ECUDA;
            }
            if (rc == CCS_OK && (best == 0 || ms < best_ms)) {
                best = cands[c];
                best_ms = ms;
            }
        }
        if (rc == CCS_OK) {
            tuned_schedule_set(dev, dmax, fits, best);
            tuned[g] = best;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == CCS_ECUDA) set_last_error("ccs_autotune: a CUDA event call failed");
    return rc;
}

}  // namespace ccs

using namespace ccs;


extern "C" size_t ccs_batch_workspace_size(const ccs_problem *probs, int32_t count) {
    if (!probs || count < 1) return 0;
    return batch_ws(probs, count);
}

static int decode_batch_impl(const ccs_problem *probs, int32_t count, const ccs_params *params,
                             ccs_result *out, void *ws, size_t ws_bytes, ccs_stream_t stream,
                             ccs_result *dev_out, cudaGraphExec_t *capture = nullptr,
                             int32_t *tuned = nullptr) {
    if (!probs || count < 1 || !out || !ws) {
        set_last_error("ccs_decode_batch: bad arguments");
        return CCS_EINVAL;
    }
    ccs_params p;
    if (params) p = *params;
    else ccs_params_init(&p);
    const size_t need = batch_ws(probs, count);
    if (need == 0) return CCS_EINVAL;
    int dmin = 16;
    for (int32_t q = 0; q < count; ++q) {
        const ccs_problem &pr = probs[q];
        if (!pr.csc_rows || !pr.csr_ptr || !pr.csr_cols || !pr.y || !pr.x_hat || !pr.r) {
            set_last_error("ccs_decode_batch: problem %d has a null pointer", q);
            return CCS_EINVAL;
        }
        dmin = pr.d < dmin ? pr.d : dmin;
    }
    int rc = check_params(&p, dmin);
    if (rc) return rc;
    if (ws_bytes < need) {
        set_last_error("ccs_decode_batch: workspace %zu < %zu bytes", ws_bytes, need);
        return CCS_ENOMEM;
    }
    if ((rc = check_aligned("ccs_decode_batch", "ws", ws, kWorkspaceAlign))) return rc;
    for (int32_t q = 0; q < count; ++q) {
        const ccs_problem &pr = probs[q];
        char who[48];
        std::snprintf(who, sizeof who, "ccs_decode_batch: problem %d", q);
        if ((rc = check_problem_arrays(who, pr.csc_rows, pr.csr_ptr, pr.csr_cols, pr.y, pr.x_hat,
                                       pr.r, pr.r0_hist)))
            return rc;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char *hdr = static_cast<char *>(ws);
    char *rhdr = hdr + engine_header_bytes(count);
    char *base = rhdr + engine_resume_header_bytes(count);
    std::vector<ProblemDev> pds(count);
    for (int32_t q = 0; q < count; ++q) {
        const ccs_problem &pr = probs[q];
        ProblemDev &P = pds[q];
        P = ProblemDev{};
        P.n = pr.n;
        P.m = pr.m;
        P.d = pr.d;
        P.csc_rows = pr.csc_rows;
        P.csr_ptr = pr.csr_ptr;
        P.csr_cols = pr.csr_cols;
        P.y = pr.y;
        P.x_hat = pr.x_hat;
        P.r = pr.r;
        P.r0_hist = pr.r0_hist;
        P.ctrl = header_ctrl(hdr, q);
        P.out_slot = q;
        base += decode_ws_layout(pr.n, pr.m, &P, base);
    }
    if (p.engine == CCS_ENGINE_HOST_LOOP) {
        if (capture) {
            set_last_error("ccs_batch_graph_create: the host-driven engine cannot be captured");
            return CCS_EINVAL;
        }
        if (dev_out) {
            set_last_error("ccs_decode_batch_async: the host-driven engine cannot run asynchronously");
            return CCS_EINVAL;
        }
        // one decode after another, each with its own launches
        for (int32_t q = 0; q < count; ++q) {
            rc = decode_host_loop(pds[q], p, &out[q], s);
            if (rc != CCS_OK) return rc;
        }
        return CCS_OK;
    }
    // A batch goes out as up to four launches, one per class, each over the
    // whole GPU: d <= 8 and d > 8 run on different kernel instances (the
    // register-resident arrays are sized by the largest d of a launch), and
    // problems whose fingerprints do not fit shared memory would shrink every
    // other problem's launch plan (fewer stages, a smaller queue) and its
    // thread count.  Every problem's result is the same either way.
    std::vector<int> cls(count);
    for (int32_t q = 0; q < count; ++q)
        cls[q] = (pds[q].d > 8 ? 2 : 0) + (engine_fp_fits(pds[q], p) ? 0 : 1);
    std::vector<int> order;
    int sizes[4] = {0, 0, 0, 0};
    int groups = 0;
    for (int c = 0; c < 4; ++c) {
        int cnt = 0;
        for (int32_t q = 0; q < count; ++q)
            if (cls[q] == c) {
                order.push_back(q);
                ++cnt;
            }
        if (cnt) sizes[groups++] = cnt;
    }
    // descriptors in launch order; each launch's control blocks sit at the
    // front of the header, and out_slot keeps the caller's index
    std::vector<ProblemDev> sub(count);
    for (int g = 0, t = 0; g < groups; ++g)
        for (int u = 0; u < sizes[g]; ++u, ++t) {
            sub[t] = pds[order[t]];
            sub[t].ctrl = header_ctrl(hdr, u);
        }
    std::vector<ccs_result> part(count);
    if (tuned) return autotune_groups(sub, sizes, groups, p, hdr, s, tuned);
    if (groups > 1) {
        // each group alone for its first iterations, then one launch over the
        // whole batch for the problems still running, so that the groups'
        // tails (problems that iterate to max_iter) overlap
        for (int t = 0; t < count; ++t) sub[t].ctrl = header_ctrl(hdr, t);
        if (capture)
            return engine_capture_phased(sub.data(), sizes, groups, count, p, kGroupIters, hdr,
                                         rhdr, dev_out, capture);
        return engine_run_phased(sub.data(), sizes, groups, count, p, kGroupIters, hdr, rhdr, s,
                                 dev_out, out);
    }
    if (capture) return engine_capture(sub.data(), sizes, groups, p, hdr, dev_out, capture);
    for (int g = 0, first = 0; g < groups; first += sizes[g], ++g) {
        rc = engine_run(sub.data() + first, sizes[g], p, part.data() + first, hdr, s, dev_out);
        if (rc != CCS_OK) return rc;
    }
    if (!dev_out)
        for (int t = 0; t < count; ++t) out[order[t]] = part[t];
    return CCS_OK;
}

extern "C" int ccs_decode_batch(const ccs_problem *probs, int32_t count, const ccs_params *params,
                                ccs_result *out, void *ws, size_t ws_bytes,
                                ccs_stream_t stream) {
    return decode_batch_impl(probs, count, params, out, ws, ws_bytes, stream, nullptr);
}

extern "C" int ccs_decode_batch_async(const ccs_problem *probs, int32_t count,
                                      const ccs_params *params, ccs_result *out_dev, void *ws,
                                      size_t ws_bytes, ccs_stream_t stream) {
    if (!out_dev) {
        set_last_error("ccs_decode_batch_async: null result pointer");
        return CCS_EINVAL;
    }
    std::vector<ccs_result> unused(count > 0 ? count : 1);
    return decode_batch_impl(probs, count, params, unused.data(), ws, ws_bytes, stream, out_dev);
}

struct ccs_graph {
    cudaGraphExec_t exec = nullptr;
};

extern "C" int ccs_batch_graph_create(const ccs_problem *probs, int32_t count,
                                      const ccs_params *params, ccs_result *out_dev, void *ws,
                                      size_t ws_bytes, ccs_graph **out) {
    if (!out || !out_dev) {
        set_last_error("ccs_batch_graph_create: null argument");
        return CCS_EINVAL;
    }
    ccs_graph *g = new ccs_graph();
    std::vector<ccs_result> unused(count > 0 ? count : 1);
    const int rc = decode_batch_impl(probs, count, params, unused.data(), ws, ws_bytes, nullptr,
                                     out_dev, &g->exec);
    if (rc != CCS_OK) {
        delete g;
        return rc;
    }
    *out = g;
    return CCS_OK;
}

extern "C" int ccs_graph_launch(ccs_graph *g, ccs_stream_t stream) {
    if (!g || !g->exec) return CCS_EINVAL;
    count_launches(1);
    CCS_CUDA_TRY(cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(stream)));
    return CCS_OK;
}

extern "C" int ccs_graph_destroy(ccs_graph *g) {
    if (!g) return CCS_EINVAL;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    delete g;
    return CCS_OK;
}

extern "C" int ccs_autotune(const ccs_problem *probs, int32_t count, const ccs_params *params,
                            void *ws, size_t ws_bytes, ccs_stream_t stream, int32_t *tuned) {
    if (!tuned) {
        set_last_error("ccs_autotune: null output");
        return CCS_EINVAL;
    }
    if (params && params->engine == CCS_ENGINE_HOST_LOOP) {
        set_last_error("ccs_autotune: tunes the persistent engine only");
        return CCS_EINVAL;
    }
    std::vector<ccs_result> unused(count > 0 ? count : 1);
    return decode_batch_impl(probs, count, params, unused.data(), ws, ws_bytes, stream, nullptr,
                             nullptr, tuned);
}

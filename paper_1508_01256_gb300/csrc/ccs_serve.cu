// ccs_serve.cu -- continuous-batching decode server.
//
// A worker thread owns one stream and runs engine rounds: each round is one
// persistent launch over every admitted request, at most `iters_per_round`
// Parallel-l0 iterations, with each request's state (x_hat, r, fingerprints,
// slot records, control block) kept on the device between rounds.  After a
// round, finished requests are retired (their state memory returns to the
// pool) and pending requests are admitted as memory and batch slots allow,
// so requests that arrive while others are on the GPU join the next round
// and their work overlaps on the device.  Results are bit-identical to a
// decode of the same request alone: every problem's iteration depends only
// on its own data.
//
// Memory: the caller hands over one device pool; the server sub-allocates
// each admitted request's state from it (first fit, 256-byte aligned) and the
// launch header once.  A request whose state can never fit is refused at
// submission (CCS_EBUDGET); one that does not fit now waits in the queue.
//
// Two kinds of request:
//  - device requests (ccs_server_submit): A, y and the outputs are caller
//    device arrays; the pool holds the decode state only;
//  - seeded requests (ccs_server_submit_seeded): the pool holds everything
//    the request keeps on the device -- A (CSC and CSR, drawn on the device
//    from the request's seed at admission), y (copied from the host at
//    admission), x_hat, r, the decode state -- so the pool bounds the HBM
//    the server uses.  When the request finishes, x_hat (and r, the ||r||_0
//    history if asked for) are copied to the caller's host buffers, and
//    only then is its memory returned to the pool and its result published.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ccs_checks.cuh"
#include "ccs_internal.cuh"

namespace ccs {

namespace {

double now_s() {
    using clk = std::chrono::steady_clock;
    static const clk::time_point t0 = clk::now();
    return std::chrono::duration<double>(clk::now() - t0).count();
}

// First-fit allocator over [0, size) with coalescing free list.
class PoolAllocator {
  public:
    explicit PoolAllocator(size_t size) : size_(size) { free_[0] = size; }
    bool alloc(size_t bytes, size_t &off) {
        bytes = align_up(bytes, 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                off = it->first;
                const size_t rest = it->second - bytes;
                free_.erase(it);
                if (rest) free_[off + bytes] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = align_up(bytes, 256);
        used_ -= bytes;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) {
            bytes += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }
    size_t used() const { return used_; }
    size_t size() const { return size_; }

  private:
    size_t size_, used_ = 0;
    std::map<size_t, size_t> free_;
};

// Pinned host staging for the nonzero lists that leave the server in one
// round (a list that does not fit is copied on its own).
constexpr size_t kStagingBytes = 32u << 20;

struct Request {
    int64_t ticket;
    ccs_problem prob;     // device arrays (for a seeded request: pool memory,
                          // filled in at admission)
    bool seeded = false;
    bool prepared = false;   // seeded: A drawn and y uploaded
    ccs_seeded_request host{};  // seeded: the caller's host buffers
    size_t state_bytes = 0, off = 0;
    bool fresh = true;
    int rounds = 0;
    double submit_s = 0, admit_s = 0, done_s = 0;
    ccs_result result{};
};

}  // namespace

}  // namespace ccs

struct ccs_server {
    ccs_server_config cfg;
    int device = 0;
    cudaStream_t stream = nullptr;
    char *pool = nullptr;
    size_t header_off = 0;
    ccs::PoolAllocator *alloc = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<ccs::Request> pending;
    std::vector<ccs::Request> inflight;
    std::unordered_map<int64_t, ccs::Request> finished;
    int64_t next_ticket = 1;
    int *host_max = nullptr;  // pinned: largest row degree per seeded request being prepared
    unsigned long long *host_cnt = nullptr;  // pinned: nonzeros of each finished seeded request
    char *staging = nullptr;  // pinned: the finished requests' nonzero lists, on their way out
    bool stop = false;
    int error = CCS_OK;
    ccs_server_stats stats{};
    std::thread worker;
};

namespace ccs {

static size_t request_state_bytes(int32_t n, int32_t m) {
    return align_up(sizeof(DecodeCtrl), 256) + decode_ws_layout(n, m, nullptr, nullptr);
}

// Pool layout of a seeded request after its decode state: CSC, CSR offsets,
// CSR columns, y, x_hat, r, the ||r||_0 history and the expander's
// generation workspace.  Returns the total bytes; with base != null fills
// the request's device pointers (and *gen_ws).
static size_t seeded_layout(int32_t n, int32_t m, int32_t d, int32_t max_iter, int64_t x_cap,
                            char *base, ccs_problem *prob, char **gen_ws, size_t *gen_bytes,
                            char **sparse = nullptr) {
    size_t off = align_up(request_state_bytes(n, m), 256);
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off = align_up(off + bytes, 256);
        return p;
    };
    char *csc = take((size_t)n * d * 4);
    char *ptr = take(((size_t)m + 1) * 8);
    char *cols = take((size_t)n * d * 4);
    char *y = take((size_t)m * 8);
    char *x = take((size_t)n * 8);
    char *r = take((size_t)m * 8);
    char *hist = take(((size_t)max_iter + 1) * 8);
    const size_t gb = ccs_workspace_size(CCS_OP_MAKE_EXPANDER, n, m, d);
    char *gw = take(gb);
    // the nonzeros of x_hat when the request asks for them: a count, then
    // x_cap indices and x_cap values
    char *sp = x_cap > 0 ? take(8 + 16 * (size_t)x_cap) : nullptr;
    if (sparse) *sparse = sp;
    if (base) {
        prob->csc_rows = reinterpret_cast<const int32_t *>(csc);
        prob->csr_ptr = reinterpret_cast<const int64_t *>(ptr);
        prob->csr_cols = reinterpret_cast<const int32_t *>(cols);
        prob->y = reinterpret_cast<const double *>(y);
        prob->x_hat = reinterpret_cast<double *>(x);
        prob->r = reinterpret_cast<double *>(r);
        prob->r0_hist = reinterpret_cast<int64_t *>(hist);
        *gen_ws = gw;
        *gen_bytes = gb;
    }
    return off;
}

// Seeded requests just admitted (indices `todo` of inflight): upload each y,
// draw each A from its seed into the pool -- every request's construction
// enqueued first, then one wait for all their largest row degrees, then the
// row sorts -- so the worker waits on the stream once per admission, not
// once per request.  rcs[q] receives each request's status.
static void prepare_seeded(ccs_server *S, const std::vector<int> &todo, std::vector<int> &rcs) {
    const int Q = (int)todo.size();
    rcs.assign(Q, CCS_OK);
    std::vector<char *> gen(Q, nullptr);
    std::vector<int *> maxdev(Q, nullptr);
    // y first: a copy from pageable memory waits for the stream, which is
    // idle now and would not be once the constructions are enqueued
    for (int q = 0; q < Q; ++q) {
        Request &R = S->inflight[todo[q]];
        const ccs_seeded_request &h = R.host;
        size_t gen_bytes = 0;
        seeded_layout(h.n, h.m, h.d, S->cfg.params.max_iter, h.x_idx ? h.x_cap : 0,
                      S->pool + R.off, &R.prob, &gen[q], &gen_bytes);
        if (cudaMemcpyAsync(const_cast<double *>(R.prob.y), h.y, (size_t)h.m * 8,
                            cudaMemcpyHostToDevice, S->stream) != cudaSuccess)
            rcs[q] = cuda_fail(cudaGetLastError(), "server: upload of y");
    }
    for (int q = 0; q < Q; ++q) {
        if (rcs[q]) continue;
        Request &R = S->inflight[todo[q]];
        const ccs_seeded_request &h = R.host;
        rcs[q] = expander_build_async(h.n, h.m, h.d, h.a_seed,
                                      const_cast<int32_t *>(R.prob.csc_rows),
                                      const_cast<int64_t *>(R.prob.csr_ptr),
                                      const_cast<int32_t *>(R.prob.csr_cols), gen[q], S->stream,
                                      &maxdev[q]);
        if (!rcs[q] && cudaMemcpyAsync(S->host_max + q, maxdev[q], sizeof(int),
                                       cudaMemcpyDeviceToHost, S->stream) != cudaSuccess)
            rcs[q] = cuda_fail(cudaGetLastError(), "server: read-back of the row degrees");
    }
    if (cudaStreamSynchronize(S->stream) != cudaSuccess) {
        const int rc = cuda_fail(cudaGetLastError(), "server: constructing A");
        for (int q = 0; q < Q; ++q) rcs[q] = rcs[q] ? rcs[q] : rc;
        return;
    }
    for (int q = 0; q < Q; ++q) {
        if (rcs[q]) continue;
        Request &R = S->inflight[todo[q]];
        rcs[q] = expander_sort_rows(R.host.m, const_cast<int64_t *>(R.prob.csr_ptr),
                                    const_cast<int32_t *>(R.prob.csr_cols), S->host_max[q],
                                    S->stream);
        if (!rcs[q]) R.prepared = true;
    }
}

// Nonzero entries of x[0, n) as (index, value) pairs, at most cap of them, in
// no particular order; *count receives how many there are.  One warp
// reservation per 32 entries.
__global__ void k_nonzeros(int32_t n, const double *__restrict__ x, int64_t *idx, double *val,
                           int64_t cap, unsigned long long *count) {
    const int lane = threadIdx.x & 31;
    for (long long j0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); j0 < n;
         j0 += (long long)gridDim.x * blockDim.x) {
        const long long j = j0 + lane;
        const double v = j < n ? x[j] : 0.0;
        const unsigned bal = __ballot_sync(0xffffffffu, v != 0.0);
        if (!bal) continue;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(count, (unsigned long long)__popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (v != 0.0) {
            const unsigned long long k = base + __popc(bal & ((1u << lane) - 1u));
            if ((long long)k < cap) {
                idx[k] = j;
                val[k] = v;
            }
        }
    }
}

// Seeded requests finished in this round: their outputs to the callers' host
// buffers.  Every request's device work (the nonzero lists) is enqueued
// first, with one wait for all counts; then the host copies.  rcs[q]
// receives each request's status.
static void deliver_seeded(ccs_server *S, std::vector<Request *> &done, std::vector<int> &rcs) {
    const int Q = (int)done.size();
    rcs.assign(Q, CCS_OK);
    std::vector<char *> sp(Q, nullptr);
    for (int q = 0; q < Q; ++q) {
        Request &R = *done[q];
        const ccs_seeded_request &h = R.host;
        if (!h.x_idx) continue;
        char *gen = nullptr;
        size_t gen_bytes = 0;
        ccs_problem unused;
        seeded_layout(h.n, h.m, h.d, S->cfg.params.max_iter, h.x_cap, S->pool + R.off, &unused,
                      &gen, &gen_bytes, &sp[q]);
        unsigned long long *cnt = reinterpret_cast<unsigned long long *>(sp[q]);
        if (cudaMemsetAsync(cnt, 0, 8, S->stream) != cudaSuccess) {
            rcs[q] = cuda_fail(cudaGetLastError(), "server: nonzero count");
            continue;
        }
        const int blocks = std::max(1, std::min(1024, (h.n + 255) / 256));
        k_nonzeros<<<blocks, 256, 0, S->stream>>>(h.n, R.prob.x_hat,
                                                  reinterpret_cast<int64_t *>(sp[q] + 8),
                                                  reinterpret_cast<double *>(sp[q] + 8 + 8 * h.x_cap),
                                                  h.x_cap, cnt);
        count_launches(1);
        if (cudaMemcpyAsync(S->host_cnt + q, cnt, 8, cudaMemcpyDeviceToHost, S->stream) !=
            cudaSuccess)
            rcs[q] = cuda_fail(cudaGetLastError(), "server: read-back of the nonzero count");
    }
    if (cudaStreamSynchronize(S->stream) != cudaSuccess) {
        const int rc = cuda_fail(cudaGetLastError(), "server: nonzero lists");
        for (int q = 0; q < Q; ++q) rcs[q] = rcs[q] ? rcs[q] : rc;
        return;
    }
    // the dense copies go straight to the callers' buffers; the nonzero
    // lists go to the server's pinned staging area first (one wait for all
    // of them), then are ordered into the callers' buffers
    std::vector<long long> stage_off(Q, -1), nnz(Q, 0), take(Q, 0);
    size_t used = 0;
    for (int q = 0; q < Q; ++q) {
        if (rcs[q]) continue;
        const Request &R = *done[q];
        const ccs_seeded_request &h = R.host;
        cudaError_t e = cudaSuccess;
        if (h.x_hat)
            e = cudaMemcpyAsync(h.x_hat, R.prob.x_hat, (size_t)h.n * 8, cudaMemcpyDeviceToHost,
                                S->stream);
        if (e == cudaSuccess && h.r)
            e = cudaMemcpyAsync(h.r, R.prob.r, (size_t)h.m * 8, cudaMemcpyDeviceToHost, S->stream);
        if (e == cudaSuccess && h.r0_hist)
            e = cudaMemcpyAsync(h.r0_hist, R.prob.r0_hist,
                                ((size_t)R.result.iterations + 1) * 8, cudaMemcpyDeviceToHost,
                                S->stream);
        if (e == cudaSuccess && h.x_idx) {
            nnz[q] = (long long)S->host_cnt[q];
            take[q] = std::min<long long>(nnz[q], h.x_cap);
            const size_t bytes = (size_t)take[q] * 16;
            if (bytes <= kStagingBytes - used) {
                stage_off[q] = (long long)used;
                if (take[q])
                    e = cudaMemcpyAsync(S->staging + used, sp[q] + 8, (size_t)take[q] * 8,
                                        cudaMemcpyDeviceToHost, S->stream);
                if (e == cudaSuccess && take[q])
                    e = cudaMemcpyAsync(S->staging + used + (size_t)take[q] * 8,
                                        sp[q] + 8 + 8 * h.x_cap, (size_t)take[q] * 8,
                                        cudaMemcpyDeviceToHost, S->stream);
                used += bytes;
            }
        }
        if (e != cudaSuccess) rcs[q] = cuda_fail(e, "server: copy of the results to the host");
    }
    if (cudaStreamSynchronize(S->stream) != cudaSuccess) {
        const int rc = cuda_fail(cudaGetLastError(), "server: copy of the results to the host");
        for (int q = 0; q < Q; ++q) rcs[q] = rcs[q] ? rcs[q] : rc;
        return;
    }
    std::vector<std::pair<int64_t, double>> pairs;
    std::vector<int64_t> ix;
    std::vector<double> vx;
    for (int q = 0; q < Q; ++q) {
        if (rcs[q] || !done[q]->host.x_idx) continue;
        const ccs_seeded_request &h = done[q]->host;
        const long long k = take[q];
        const int64_t *pi;
        const double *pv;
        if (stage_off[q] >= 0) {  // staged
            pi = reinterpret_cast<const int64_t *>(S->staging + stage_off[q]);
            pv = reinterpret_cast<const double *>(S->staging + stage_off[q] + (size_t)k * 8);
        } else {  // larger than the staging area: straight copies
            ix.resize((size_t)k);
            vx.resize((size_t)k);
            char *gen = nullptr;
            size_t gen_bytes = 0;
            ccs_problem unused;
            char *spq = nullptr;
            seeded_layout(h.n, h.m, h.d, S->cfg.params.max_iter, h.x_cap, S->pool + done[q]->off,
                          &unused, &gen, &gen_bytes, &spq);
            cudaError_t e = cudaMemcpy(ix.data(), spq + 8, (size_t)k * 8, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess)
                e = cudaMemcpy(vx.data(), spq + 8 + 8 * h.x_cap, (size_t)k * 8,
                               cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) {
                rcs[q] = cuda_fail(e, "server: copy of the nonzeros to the host");
                continue;
            }
            pi = ix.data();
            pv = vx.data();
        }
        // ascending indices (the device list has no order)
        pairs.resize((size_t)k);
        for (long long t = 0; t < k; ++t) pairs[(size_t)t] = {pi[t], pv[t]};
        std::sort(pairs.begin(), pairs.end());
        for (long long t = 0; t < k; ++t) {
            h.x_idx[t] = pairs[(size_t)t].first;
            h.x_val[t] = pairs[(size_t)t].second;
        }
        *h.x_nnz = nnz[q];
    }
}

static void worker_loop(ccs_server *S) {
    cudaSetDevice(S->device);
    const int maxb = S->cfg.max_batch;
    std::vector<ProblemDev> pds;
    std::vector<ccs_result> res(maxb);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            // admit pending requests in arrival order while memory and slots allow
            for (auto it = S->pending.begin();
                 it != S->pending.end() && (int)S->inflight.size() < maxb;) {
                size_t off;
                if (S->alloc->alloc(it->state_bytes, off)) {
                    it->off = off;
                    it->admit_s = now_s();
                    S->inflight.push_back(*it);
                    it = S->pending.erase(it);
                    S->stats.admitted += 1;
                } else {
                    break;  // first come, first served: no overtaking
                }
            }
            if (S->inflight.empty()) {
                if (S->stop) return;
                S->cv_work.wait(lk, [&] { return S->stop || !S->pending.empty(); });
                continue;
            }
            const int64_t bytes = (int64_t)S->alloc->used();
            if (bytes > S->stats.peak_bytes) S->stats.peak_bytes = bytes;
            if ((int64_t)S->inflight.size() > S->stats.peak_inflight)
                S->stats.peak_inflight = (int64_t)S->inflight.size();
        }
        // seeded requests admitted just now: A drawn from the seed, y uploaded.
        // One that fails finishes with its error and leaves the round.
        {
            std::vector<int> todo, rcs;
            for (size_t q = 0; q < S->inflight.size(); ++q)
                if (S->inflight[q].seeded && !S->inflight[q].prepared) todo.push_back((int)q);
            if (!todo.empty()) prepare_seeded(S, todo, rcs);
            std::vector<Request> failed;
            for (int q = (int)todo.size() - 1; q >= 0; --q) {
                if (rcs[q] == CCS_OK) continue;
                Request &R = S->inflight[todo[q]];
                R.result = ccs_result{};
                R.result.error = rcs[q];
                failed.push_back(R);
                S->inflight.erase(S->inflight.begin() + todo[q]);
            }
            if (!failed.empty()) {
                std::lock_guard<std::mutex> lk(S->mu);
                const double t = now_s();
                for (Request &R : failed) {
                    R.done_s = t;
                    S->alloc->release(R.off, R.state_bytes);
                    S->finished[R.ticket] = R;
                    S->stats.completed += 1;
                }
                S->cv_done.notify_all();
                if (S->inflight.empty()) continue;
            }
        }
        // build this round's problem list (the worker alone touches inflight
        // entries' device state; submitters only append to `pending`)
        const int P = (int)S->inflight.size();
        pds.assign(P, ProblemDev{});
        int rc = CCS_OK;
        for (int p = 0; p < P && rc == CCS_OK; ++p) {
            Request &R = S->inflight[p];
            ProblemDev &D = pds[p];
            D.n = R.prob.n;
            D.m = R.prob.m;
            D.d = R.prob.d;
            D.csc_rows = R.prob.csc_rows;
            D.csr_ptr = R.prob.csr_ptr;
            D.csr_cols = R.prob.csr_cols;
            D.y = R.prob.y;
            D.x_hat = R.prob.x_hat;
            D.r = R.prob.r;
            D.r0_hist = R.prob.r0_hist;
            char *base = S->pool + R.off;
            D.ctrl = reinterpret_cast<DecodeCtrl *>(base);
            decode_ws_layout(D.n, D.m, &D, base + align_up(sizeof(DecodeCtrl), 256));
            D.flags = R.fresh ? kPdFresh : 0;
            D.out_slot = p;
            if (R.fresh && cudaMemsetAsync(D.ctrl, 0, sizeof(DecodeCtrl), S->stream) != cudaSuccess)
                rc = CCS_ECUDA;
        }
        if (rc == CCS_OK)
            rc = engine_resume(pds.data(), P, S->cfg.params, S->cfg.iters_per_round, res.data(),
                               S->pool + S->header_off, S->stream);
        // finished seeded requests hand their outputs to the host before their
        // memory returns to the pool (outside the lock: it waits on the stream)
        std::vector<int> deliver_rc(P, CCS_OK);
        {
            std::vector<Request *> fin;
            std::vector<int> at, rcs;
            for (int p = 0; p < P; ++p) {
                Request &R = S->inflight[p];
                const bool done = rc != CCS_OK || res[p].status != kRunning || res[p].error;
                if (done && R.seeded && rc == CCS_OK) {
                    R.result = res[p];
                    fin.push_back(&R);
                    at.push_back(p);
                }
            }
            if (!fin.empty()) deliver_seeded(S, fin, rcs);
            for (size_t q = 0; q < at.size(); ++q) deliver_rc[at[q]] = rcs[q];
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stats.rounds += 1;
            std::vector<Request> keep;
            keep.reserve(P);
            const double t = now_s();
            for (int p = 0; p < P; ++p) {
                Request &R = S->inflight[p];
                R.rounds += 1;
                R.fresh = false;
                const bool done = rc != CCS_OK || res[p].status != kRunning || res[p].error;
                if (done) {
                    R.result = res[p];
                    if (rc != CCS_OK) R.result.error = rc;
                    else if (deliver_rc[p] != CCS_OK) R.result.error = deliver_rc[p];
                    R.done_s = t;
                    S->alloc->release(R.off, R.state_bytes);
                    S->finished[R.ticket] = R;
                    S->stats.completed += 1;
                } else {
                    keep.push_back(R);
                }
            }
            S->inflight.swap(keep);
            if (rc != CCS_OK) S->error = rc;
        }
        S->cv_done.notify_all();
    }
}

}  // namespace ccs

using namespace ccs;

extern "C" int ccs_server_create(const ccs_server_config *cfg, ccs_stream_t stream,
                                 ccs_server **out) {
    if (!cfg || !out || !cfg->pool || cfg->max_batch < 1 || cfg->max_batch > 4096 ||
        cfg->iters_per_round < 1) {
        set_last_error("ccs_server_create: bad configuration");
        return CCS_EINVAL;
    }
    if (reinterpret_cast<uintptr_t>(cfg->pool) & 255u) {
        set_last_error("ccs_server_create: the pool must start on a 256-byte boundary");
        return CCS_EINVAL;
    }
    const size_t hdr = align_up(engine_resume_header_bytes(cfg->max_batch), 256);
    if (cfg->pool_bytes < hdr + 256) {
        set_last_error("ccs_server_create: pool of %zu bytes cannot hold the %zu-byte launch header",
                       cfg->pool_bytes, hdr);
        return CCS_EBUDGET;
    }
    ccs_server *S = new ccs_server();
    S->cfg = *cfg;
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        delete S;
        return cuda_fail(cudaGetLastError(), "cudaGetDevice");
    }
    S->stream = reinterpret_cast<cudaStream_t>(stream);
    S->pool = static_cast<char *>(cfg->pool);
    // launch header at the top of the pool, on a 256-byte boundary whatever
    // pool_bytes is (its sync word and descriptors are accessed atomically)
    S->header_off = (cfg->pool_bytes - hdr) & ~(size_t)255;
    S->alloc = new PoolAllocator(S->header_off);
    if (cudaHostAlloc(reinterpret_cast<void **>(&S->host_max), sizeof(int) * cfg->max_batch,
                      cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void **>(&S->host_cnt),
                      sizeof(unsigned long long) * cfg->max_batch,
                      cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void **>(&S->staging), kStagingBytes,
                      cudaHostAllocDefault) != cudaSuccess) {
        if (S->host_max) cudaFreeHost(S->host_max);
        if (S->host_cnt) cudaFreeHost(S->host_cnt);
        delete S->alloc;
        delete S;
        return cuda_fail(cudaGetLastError(), "ccs_server_create: pinned host buffer");
    }
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return CCS_OK;
}

extern "C" int ccs_server_submit(ccs_server *S, const ccs_problem *req, int64_t *ticket) {
    if (!S || !req || !ticket) {
        set_last_error("ccs_server_submit: null argument");
        return CCS_EINVAL;
    }
    int rc = check_sizes(req->n, req->m, req->d);
    if (rc) return rc;
    if ((rc = check_params(&S->cfg.params, req->d))) return rc;
    if (!req->csc_rows || !req->csr_ptr || !req->csr_cols || !req->y || !req->x_hat || !req->r) {
        set_last_error("ccs_server_submit: null array");
        return CCS_EINVAL;
    }
    if ((rc = check_problem_arrays("ccs_server_submit", req->csc_rows, req->csr_ptr,
                                   req->csr_cols, req->y, req->x_hat, req->r, req->r0_hist)))
        return rc;
    Request R;
    R.prob = *req;
    R.state_bytes = request_state_bytes(req->n, req->m);
    if (align_up(R.state_bytes, 256) > S->alloc->size()) {
        set_last_error("ccs_server_submit: request needs %zu bytes of state, pool holds %zu",
                       R.state_bytes, S->alloc->size());
        return CCS_EBUDGET;
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) {
            set_last_error("ccs_server_submit: server is shutting down");
            return CCS_EBUSY;
        }
        R.ticket = S->next_ticket++;
        R.submit_s = now_s();
        S->pending.push_back(R);
        S->stats.submitted += 1;
        *ticket = R.ticket;
    }
    S->cv_work.notify_one();
    return CCS_OK;
}

extern "C" size_t ccs_seeded_request_bytes(int32_t n, int32_t m, int32_t d, int32_t max_iter,
                                           int64_t x_cap) {
    if (check_sizes(n, m, d) != CCS_OK || max_iter < 0 || x_cap < 0) return 0;
    return seeded_layout(n, m, d, max_iter, x_cap, nullptr, nullptr, nullptr, nullptr);
}

extern "C" int ccs_server_submit_seeded(ccs_server *S, const ccs_seeded_request *req,
                                        int64_t *ticket) {
    if (!S || !req || !ticket) {
        set_last_error("ccs_server_submit_seeded: null argument");
        return CCS_EINVAL;
    }
    int rc = check_sizes(req->n, req->m, req->d);
    if (rc) return rc;
    if ((rc = check_params(&S->cfg.params, req->d))) return rc;
    const bool sparse = req->x_idx || req->x_val || req->x_nnz;
    if (!req->y || (!req->x_hat && !sparse) ||
        (sparse && (!req->x_idx || !req->x_val || !req->x_nnz || req->x_cap < 1))) {
        set_last_error("ccs_server_submit_seeded: need y and x_hat, or x_idx, x_val, x_nnz and "
                       "x_cap >= 1");
        return CCS_EINVAL;
    }
    Request R;
    R.seeded = true;
    R.host = *req;
    R.prob.n = req->n;
    R.prob.m = req->m;
    R.prob.d = req->d;
    R.state_bytes = seeded_layout(req->n, req->m, req->d, S->cfg.params.max_iter,
                                  sparse ? req->x_cap : 0, nullptr, nullptr, nullptr, nullptr);
    if (R.state_bytes > S->alloc->size()) {
        set_last_error("ccs_server_submit_seeded: request needs %zu bytes, pool holds %zu",
                       R.state_bytes, S->alloc->size());
        return CCS_EBUDGET;
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) {
            set_last_error("ccs_server_submit_seeded: server is shutting down");
            return CCS_EBUSY;
        }
        R.ticket = S->next_ticket++;
        R.submit_s = now_s();
        S->pending.push_back(R);
        S->stats.submitted += 1;
        *ticket = R.ticket;
    }
    S->cv_work.notify_one();
    return CCS_OK;
}

static void fill_info(const Request &R, ccs_ticket_info *info) {
    info->result = R.result;
    info->submit_s = R.submit_s;
    info->admit_s = R.admit_s;
    info->done_s = R.done_s;
    info->rounds = R.rounds;
    info->reserved = 0;
}

extern "C" int ccs_server_poll(ccs_server *S, int64_t ticket, ccs_ticket_info *info) {
    if (!S || !info) return CCS_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->finished.find(ticket);
    if (it == S->finished.end()) {
        if (ticket <= 0 || ticket >= S->next_ticket) {
            set_last_error("ccs_server_poll: unknown ticket %lld", (long long)ticket);
            return CCS_EINVAL;
        }
        return CCS_EBUSY;
    }
    fill_info(it->second, info);
    S->finished.erase(it);
    return CCS_OK;
}

extern "C" int ccs_server_wait(ccs_server *S, int64_t ticket, ccs_ticket_info *info,
                               int32_t timeout_ms) {
    if (!S || !info) return CCS_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    if (ticket <= 0 || ticket >= S->next_ticket) {
        set_last_error("ccs_server_wait: unknown ticket %lld", (long long)ticket);
        return CCS_EINVAL;
    }
    const auto ready = [&] { return S->finished.count(ticket) != 0; };
    if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms), ready))
        return CCS_EBUSY;
    auto it = S->finished.find(ticket);
    fill_info(it->second, info);
    S->finished.erase(it);
    return CCS_OK;
}

extern "C" int ccs_server_stats_get(ccs_server *S, ccs_server_stats *out) {
    if (!S || !out) return CCS_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->stats;
    out->bytes_in_use = (int64_t)S->alloc->used();
    out->pending = (int64_t)S->pending.size();
    out->inflight = (int64_t)S->inflight.size();
    out->error = S->error;
    return CCS_OK;
}

extern "C" int ccs_server_destroy(ccs_server *S) {
    if (!S) return CCS_EINVAL;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    const int err = S->error;
    cudaFreeHost(S->host_max);
    cudaFreeHost(S->host_cnt);
    cudaFreeHost(S->staging);
    delete S->alloc;
    delete S;
    return err;
}

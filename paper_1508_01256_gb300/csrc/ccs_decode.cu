// ccs_decode.cu -- the Parallel-l0 iteration (Alg. 2) on one problem.
//
// One iteration is two kernels:
//   score   every column j reads r on its d rows (held in registers), finds
//           the most frequent nonzero value omega_j (ties: the smallest),
//           scores it (Eq. (15): c_omega - c_0, or Alg. 8: c_omega) and, if
//           accepted, applies x_hat_j += omega_j at once (each column owns
//           its x_hat_j, so the updates of one iteration do not interact).
//           It also marks the rows N(j) as touched and, the first time a
//           column becomes nonzero, enters j in the contributor slots of its
//           rows.
//   residual every touched row recomputes r_i = y_i - sum over its nonzero
//           x_hat_j in ascending j, from +0.0.  Rows not touched keep r_i:
//           none of their columns changed, so the same ordered sum would
//           give the same bits.  The change of ||r||_0 is summed exactly in
//           integers.
// A one-thread kernel then applies the stop rule (||r||_0 == 0, nothing
// accepted, or max_iter) and records ||r||_0.
#include "ccs_checks.cuh"
#include "ccs_device.cuh"

namespace ccs {

// ---- init --------------------------------------------------------------

__global__ void k_init(ProblemDev P) {
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long nz = 0;
    for (long long j = tid; j < P.n; j += stride) {
        P.x_hat[j] = 0.0;
        P.in_slots[j] = 0;
    }
    for (long long i = tid; i < P.m; i += stride) {
        const double v = P.y[i];
        P.r[i] = v;
        store_fp(P, i, v);
        P.touched[i] = 0;
        P.slots[(size_t)i * kSlotRec] = 0;
        nz += (v != 0.0);
    }
    nz = warp_sum_ll(nz);
    if ((threadIdx.x & 31) == 0 && nz)
        atomicAdd(reinterpret_cast<unsigned long long *>(&P.ctrl->r0), (unsigned long long)nz);
}

__global__ void k_init_finish(ProblemDev P, int max_iter) {
    DecodeCtrl *c = P.ctrl;
    c->iteration = 0;
    c->max_iter = max_iter;
    if (P.r0_hist) P.r0_hist[0] = c->r0;
    c->status = (c->r0 == 0) ? CCS_CONVERGED : (max_iter == 0 ? CCS_MAX_ITER : kRunning);
}

// ---- score + apply ------------------------------------------------------

template <int D>
__global__ void __launch_bounds__(256) k_score(ProblemDev P, int alpha, int mode) {
    if (ld_volatile(&P.ctrl->status) != kRunning) return;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    bool acc = false;
    if (j < P.n) {
        int32_t rows[D];
#pragma unroll
        for (int t = 0; t < D; ++t) rows[t] = __ldg(P.csc_rows + (size_t)j * D + t);
        unsigned long long omega;
        acc = exact_score<D>(rows, D, P.r, alpha, mode, &omega);
        if (acc) apply_pair<D>(P, j, rows, D, omega);
    }
    // block total on chip, then one global atomic per block
    __shared__ unsigned s_acc;
    if (threadIdx.x == 0) s_acc = 0;
    __syncthreads();
    const unsigned bal = __ballot_sync(0xffffffffu, acc);
    if ((threadIdx.x & 31) == 0 && bal) atomicAdd(&s_acc, (unsigned)__popc(bal));
    __syncthreads();
    if (threadIdx.x == 0 && s_acc)
        atomicAdd(&P.ctrl->acc[P.ctrl->iteration & 3], (unsigned long long)s_acc);
}

// ---- residual + ||r||_0 ---------------------------------------------------

__global__ void __launch_bounds__(256) k_residual(ProblemDev P) {
    if (ld_volatile(&P.ctrl->status) != kRunning) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    long long delta = 0;
    bool touched = false, over = false;
    int js[kSlotRec];
    double s = 0.0;
    if (i < P.m && P.touched[i]) {
        touched = true;
        load_record(P, i, js);
        over = js[0] > kSlots;
        if (!over) s = row_sum_from_record(P, i, js);
    }
    const double so = overflow_row_sums(P, over, i, lane);  // whole warp
    if (touched) {
        if (over) s = so;
        P.touched[i] = 0;
        const double rn = __dsub_rn(P.y[i], s);
        const double ro = P.r[i];
        delta = (long long)(rn != 0.0) - (long long)(ro != 0.0);
        P.r[i] = rn;
        store_fp(P, i, rn);
    }
    __shared__ long long s_delta;
    if (threadIdx.x == 0) s_delta = 0;
    __syncthreads();
    delta = warp_sum_ll(delta);
    if ((threadIdx.x & 31) == 0 && delta)
        atomicAdd(reinterpret_cast<unsigned long long *>(&s_delta), (unsigned long long)delta);
    __syncthreads();
    if (threadIdx.x == 0 && s_delta)
        atomicAdd(reinterpret_cast<unsigned long long *>(&P.ctrl->r0), (unsigned long long)s_delta);
}

// ---- stop rule --------------------------------------------------------------

__global__ void k_finish(ProblemDev P) {
    DecodeCtrl *c = P.ctrl;
    if (c->status != kRunning) return;
    const int slot = c->iteration & 3;
    if (c->acc[slot] == 0) {
        c->status = CCS_STALLED;
        return;
    }
    c->acc[slot] = 0;
    c->iteration += 1;
    if (P.r0_hist) P.r0_hist[c->iteration] = c->r0;
    if (c->r0 == 0) c->status = CCS_CONVERGED;
    else if (c->iteration >= c->max_iter) c->status = CCS_MAX_ITER;
}

// ---- dispatch ----------------------------------------------------------------

typedef void (*score_fn)(ProblemDev, int, int);

static score_fn score_kernel(int d) {
    switch (d) {
        case 1: return k_score<1>;
        case 2: return k_score<2>;
        case 3: return k_score<3>;
        case 4: return k_score<4>;
        case 5: return k_score<5>;
        case 6: return k_score<6>;
        case 7: return k_score<7>;
        case 8: return k_score<8>;
        case 9: return k_score<9>;
        case 10: return k_score<10>;
        case 11: return k_score<11>;
        case 12: return k_score<12>;
        case 13: return k_score<13>;
        case 14: return k_score<14>;
        case 15: return k_score<15>;
        case 16: return k_score<16>;
        default: return nullptr;
    }
}

int check_params(const ccs_params *p, int d) {
    if (p->alpha < 2 || p->alpha > d) {
        set_last_error("alpha=%d outside [2, d=%d]", p->alpha, d);
        return CCS_EINVAL;
    }
    if (p->max_iter < 0) {
        set_last_error("max_iter=%d < 0", p->max_iter);
        return CCS_EINVAL;
    }
    if (p->score_mode != CCS_SCORE_L0_DECREASE && p->score_mode != CCS_SCORE_COUNT) {
        set_last_error("unknown score_mode %d", p->score_mode);
        return CCS_EINVAL;
    }
    if (p->engine != CCS_ENGINE_AUTO && p->engine != CCS_ENGINE_HOST_LOOP &&
        p->engine != CCS_ENGINE_PERSISTENT) {
        set_last_error("unknown engine %d", p->engine);
        return CCS_EINVAL;
    }
    const int stage_cap = (p->schedule >> 2) & 7;
    if (p->watchdog_ms < 0 || p->schedule < 0 || p->schedule >= 128 || stage_cap == 1 ||
        stage_cap > 6 || ((p->schedule >> 5) & 3) == 3) {
        set_last_error("bad watchdog_ms or schedule (%d)", p->schedule);
        return CCS_EINVAL;
    }
    if (p->shifted != 0 && p->shifted != 1) {
        set_last_error("shifted must be 0 or 1 (got %d)", p->shifted);
        return CCS_EINVAL;
    }
    if (p->shifted && p->engine == CCS_ENGINE_HOST_LOOP) {
        set_last_error("the shifted variant runs on the persistent engine only");
        return CCS_EINVAL;
    }
    return CCS_OK;
}

// Host-driven loop: one score, residual and stop-rule launch per iteration,
// then a 64-byte read of the control block to decide whether to go on.
int decode_host_loop(const ProblemDev &P, const ccs_params &p, ccs_result *out,
                     cudaStream_t s) {
    score_fn score = score_kernel(P.d);
    const int nb_cols = (P.n + 255) / 256, nb_rows = (P.m + 255) / 256;
    const long long big = P.n > P.m ? P.n : P.m;
    const int nb_init = (int)((big + 255) / 256 < 152 * 16 ? (big + 255) / 256 : 152 * 16);
    CCS_CUDA_TRY(cudaMemsetAsync(P.ctrl, 0, sizeof(DecodeCtrl), s));
    int ev = prof_start(CCS_K_INIT, s);
    k_init<<<nb_init, 256, 0, s>>>(P);
    prof_stop(ev, s);
    k_init_finish<<<1, 1, 0, s>>>(P, p.max_iter);
    count_launches(2);
    CCS_CUDA_TRY(cudaGetLastError());
    DecodeCtrl h;
    CCS_CUDA_TRY(cudaMemcpyAsync(&h, P.ctrl, sizeof(h), cudaMemcpyDeviceToHost, s));
    CCS_CUDA_TRY(cudaStreamSynchronize(s));
    while (h.status == kRunning) {
        ev = prof_start(CCS_K_SCORE, s);
        score<<<nb_cols, 256, 0, s>>>(P, p.alpha, p.score_mode);
        prof_stop(ev, s);
        ev = prof_start(CCS_K_RESIDUAL, s);
        k_residual<<<nb_rows, 256, 0, s>>>(P);
        prof_stop(ev, s);
        ev = prof_start(CCS_K_FINISH, s);
        k_finish<<<1, 1, 0, s>>>(P);
        prof_stop(ev, s);
        count_launches(3);
        CCS_CUDA_TRY(cudaGetLastError());
        CCS_CUDA_TRY(cudaMemcpyAsync(&h, P.ctrl, sizeof(h), cudaMemcpyDeviceToHost, s));
        CCS_CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (profiling()) prof_collect();
    out->status = h.status;
    out->iterations = h.iteration;
    out->r0_final = h.r0;
    out->error = (h.error & kErrWatchdog) ? CCS_ETIMEOUT : CCS_OK;
    out->row_driven = 0;
    out->row_entries = 0;
    out->residual_form = CCS_RESIDUAL_ORDERED;
    out->reserved = 0;
    return out->error;
}


// Shared set-up of the blocking and asynchronous single-problem calls.
static int decode_setup(int32_t n, int32_t m, int32_t d, const int32_t *csc_rows,
                        const int64_t *csr_ptr, const int32_t *csr_cols, const double *y,
                        double *x_hat, double *r, int64_t *r0_hist, const ccs_params *params,
                        void *out, void *ws, size_t ws_bytes, const char *who, ccs_params &p,
                        ProblemDev &P) {
    int rc = check_sizes(n, m, d);
    if (rc) return rc;
    if (params) p = *params;
    else ccs_params_init(&p);
    if ((rc = check_params(&p, d))) return rc;
    if (!csc_rows || !csr_ptr || !csr_cols || !y || !x_hat || !r || !out || !ws) {
        set_last_error("%s: null pointer argument", who);
        return CCS_EINVAL;
    }
    const size_t need = engine_header_bytes(1) + decode_ws_layout(n, m, nullptr, nullptr);
    if (ws_bytes < need) {
        set_last_error("%s: workspace %zu < %zu bytes", who, ws_bytes, need);
        return CCS_ENOMEM;
    }
    if ((rc = check_problem_arrays(who, csc_rows, csr_ptr, csr_cols, y, x_hat, r, r0_hist)) ||
        (rc = check_aligned(who, "ws", ws, kWorkspaceAlign)))
        return rc;
    P = ProblemDev{};
    P.n = n;
    P.m = m;
    P.d = d;
    P.csc_rows = csc_rows;
    P.csr_ptr = csr_ptr;
    P.csr_cols = csr_cols;
    P.y = y;
    P.x_hat = x_hat;
    P.r = r;
    P.r0_hist = r0_hist;
    char *base = static_cast<char *>(ws);
    P.ctrl = header_ctrl(base, 0);
    decode_ws_layout(n, m, &P, base + engine_header_bytes(1));
    return CCS_OK;
}

}  // namespace ccs

using namespace ccs;

extern "C" int ccs_decode_parallel_l0(int32_t n, int32_t m, int32_t d, const int32_t *csc_rows,
                                      const int64_t *csr_ptr, const int32_t *csr_cols,
                                      const double *y, double *x_hat, double *r,
                                      int64_t *r0_hist, const ccs_params *params,
                                      ccs_result *out, void *ws, size_t ws_bytes,
                                      ccs_stream_t stream) {
    ccs_params p;
    ProblemDev P;
    int rc = decode_setup(n, m, d, csc_rows, csr_ptr, csr_cols, y, x_hat, r, r0_hist, params, out,
                          ws, ws_bytes, "ccs_decode_parallel_l0", p, P);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (p.engine == CCS_ENGINE_HOST_LOOP) return decode_host_loop(P, p, out, s);
    return engine_run(&P, 1, p, out, static_cast<char *>(ws), s);
}

extern "C" int ccs_decode_parallel_l0_async(int32_t n, int32_t m, int32_t d,
                                            const int32_t *csc_rows, const int64_t *csr_ptr,
                                            const int32_t *csr_cols, const double *y,
                                            double *x_hat, double *r, int64_t *r0_hist,
                                            const ccs_params *params, ccs_result *out_dev,
                                            void *ws, size_t ws_bytes, ccs_stream_t stream) {
    ccs_params p;
    ProblemDev P;
    int rc = decode_setup(n, m, d, csc_rows, csr_ptr, csr_cols, y, x_hat, r, r0_hist, params,
                          out_dev, ws, ws_bytes, "ccs_decode_parallel_l0_async", p, P);
    if (rc) return rc;
    if (p.engine == CCS_ENGINE_HOST_LOOP) {
        set_last_error("ccs_decode_parallel_l0_async: the host-driven engine cannot run asynchronously");
        return CCS_EINVAL;
    }
    ccs_result unused;
    return engine_run(&P, 1, p, &unused, static_cast<char *>(ws),
                      reinterpret_cast<cudaStream_t>(stream), out_dev);
}

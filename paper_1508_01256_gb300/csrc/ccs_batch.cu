// ccs_batch.cu -- many independent decodes per call.
#include <vector>

#include "ccs_internal.cuh"

namespace ccs {

static size_t batch_ws(const ccs_problem *probs, int32_t count) {
    size_t total = 0;
    for (int32_t q = 0; q < count; ++q) {
        if (check_sizes(probs[q].n, probs[q].m, probs[q].d) != CCS_OK) return 0;
        total += decode_ws_layout(probs[q].n, probs[q].m, nullptr, nullptr);
    }
    return total;
}

}  // namespace ccs

using namespace ccs;

extern "C" size_t ccs_batch_workspace_size(const ccs_problem *probs, int32_t count) {
    if (!probs || count < 1) return 0;
    return batch_ws(probs, count);
}

extern "C" int ccs_decode_batch(const ccs_problem *probs, int32_t count, const ccs_params *params,
                                ccs_result *out, void *ws, size_t ws_bytes,
                                ccs_stream_t stream) {
    if (!probs || count < 1 || !out || !ws) {
        set_last_error("ccs_decode_batch: bad arguments");
        return CCS_EINVAL;
    }
    const size_t need = batch_ws(probs, count);
    if (need == 0) return CCS_EINVAL;
    if (ws_bytes < need) {
        set_last_error("ccs_decode_batch: workspace %zu < %zu bytes", ws_bytes, need);
        return CCS_ENOMEM;
    }
    char *base = static_cast<char *>(ws);
    for (int32_t q = 0; q < count; ++q) {
        const ccs_problem &pr = probs[q];
        const size_t bytes = decode_ws_layout(pr.n, pr.m, nullptr, nullptr);
        int rc = ccs_decode_parallel_l0(pr.n, pr.m, pr.d, pr.csc_rows, pr.csr_ptr, pr.csr_cols,
                                        pr.y, pr.x_hat, pr.r, pr.r0_hist, params, &out[q], base,
                                        bytes, stream);
        if (rc != CCS_OK && rc != CCS_ETIMEOUT) return rc;
        base += bytes;
    }
    return CCS_OK;
}

// ccs_noalloc.cu -- Parallel-l0 decode that allocates nothing.
//
// Some callers cannot allocate device memory at the moment they decode: code
// running under a fixed memory budget that is already fully reserved,
// real-time loops where an allocation (and the synchronisation it can cause)
// is not allowed, or hosts that only hand out pre-registered buffers.  They
// still own the inputs and outputs, but cannot supply a workspace.  For them
// this file keeps the decode's scratch in one statically sized device array
// that belongs to the library: every GPU that loads the library holds it
// until the process exits.
//
// Host code never uses the array's name as a device address (in host code it
// names a host-side stand-in).  Instead, once per device and with that device
// current, cudaGetSymbolAddress gives the real device address, which is
// cached and passed to the kernel.  The cached address belongs to the
// device's context as it was at that first call: after cudaDeviceReset the
// module is loaded again and the address may change, so calls after a reset
// are not supported.
#include <mutex>

#include "ccs_internal.cuh"

namespace ccs {

// Largest workspace the static scratch can stand in for.
constexpr size_t kNoAllocScratchBytes = 16u << 20;  // 16 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocDevices = 64;

// Device address of g_noalloc_scratch on the current device (set up on the
// first call on each device).  Returns CCS_OK or an error code.
static int scratch_address(void **out) {
    static std::mutex mu;
    static void *addr[kNoAllocDevices];
    int dev = 0;
    CCS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocDevices) {
        set_last_error("ccs_decode_parallel_l0_noalloc: device %d beyond the supported %d", dev,
                       kNoAllocDevices);
        return CCS_EINVAL;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        addr[dev] = p;
    }
    *out = addr[dev];
    return CCS_OK;
}

}  // namespace ccs

using namespace ccs;

extern "C" size_t ccs_noalloc_scratch_bytes(void) { return kNoAllocScratchBytes; }

extern "C" int ccs_decode_parallel_l0_noalloc(int32_t n, int32_t m, int32_t d,
                                              const int32_t *csc_rows, const int64_t *csr_ptr,
                                              const int32_t *csr_cols, const double *y,
                                              double *x_hat, double *r, int64_t *r0_hist,
                                              const ccs_params *params, ccs_result *out,
                                              ccs_stream_t stream) {
    int rc = check_sizes(n, m, d);
    if (rc) return rc;
    const size_t need = ccs_workspace_size(CCS_OP_DECODE, n, m, d);
    if (need > kNoAllocScratchBytes) {
        set_last_error("ccs_decode_parallel_l0_noalloc: n=%d, m=%d need %zu bytes of scratch, "
                       "more than the %zu bytes kept for this entry point",
                       n, m, need, kNoAllocScratchBytes);
        return CCS_EINVAL;
    }
    ccs_params p;
    if (params) p = *params;
    else ccs_params_init(&p);
    if (p.engine == CCS_ENGINE_HOST_LOOP) {
        set_last_error("ccs_decode_parallel_l0_noalloc: runs on the persistent engine only");
        return CCS_EINVAL;
    }
    void *scratch = nullptr;
    if ((rc = scratch_address(&scratch))) return rc;
    // The scratch keeps the previous call's contents; the decode clears what
    // must start at zero (barrier word and control block by memset, the rest
    // in its own init phase), exactly as with a caller workspace.
    return ccs_decode_parallel_l0(n, m, d, csc_rows, csr_ptr, csr_cols, y, x_hat, r, r0_hist,
                                  &p, out, scratch, kNoAllocScratchBytes, stream);
}

// ccs_engine_k512_d11_12.cu -- persistent engine kernel instances
// k_engine<11, 512> and k_engine<12, 512>.
#include "ccs_engine_kernel.cuh"

namespace ccs {

engine_fn engine_kernel_512_d11(int dmax) {
    return dmax == 11 ? k_engine<11, 512> : k_engine<12, 512>;
}

}  // namespace ccs

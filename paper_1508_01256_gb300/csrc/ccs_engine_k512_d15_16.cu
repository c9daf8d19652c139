// ccs_engine_k512_d15_16.cu -- persistent engine kernel instances
// k_engine<15, 512> and k_engine<16, 512>.
#include "ccs_engine_kernel.cuh"

namespace ccs {

engine_fn engine_kernel_512_d15(int dmax) {
    return dmax == 15 ? k_engine<15, 512> : k_engine<16, 512>;
}

}  // namespace ccs

// ccs_engine_k512_d3_4.cu -- persistent engine kernel instances
// k_engine<3, 512> and k_engine<4, 512>.
#include "ccs_engine_kernel.cuh"

namespace ccs {

engine_fn engine_kernel_512_d3(int dmax) {
    return dmax == 3 ? k_engine<3, 512> : k_engine<4, 512>;
}

}  // namespace ccs

// ccs_engine_k1024_d3_4.cu -- persistent engine kernel instances
// k_engine<3, 1024> and k_engine<4, 1024>.
#include "ccs_engine_kernel.cuh"

namespace ccs {

engine_fn engine_kernel_1024_d3(int dmax) {
    return dmax == 3 ? k_engine<3, 1024> : k_engine<4, 1024>;
}

}  // namespace ccs

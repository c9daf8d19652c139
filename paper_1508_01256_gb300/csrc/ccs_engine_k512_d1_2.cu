// ccs_engine_k512_d1_2.cu -- persistent engine kernel instances
// k_engine<1, 512> and k_engine<2, 512>.
#include "ccs_engine_kernel.cuh"

namespace ccs {

engine_fn engine_kernel_512_d1(int dmax) {
    return dmax == 1 ? k_engine<1, 512> : k_engine<2, 512>;
}

}  // namespace ccs

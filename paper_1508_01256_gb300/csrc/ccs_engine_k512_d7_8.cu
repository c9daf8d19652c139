// ccs_engine_k512_d7_8.cu -- persistent engine kernel instances
// k_engine<7, 512> and k_engine<8, 512>.
#include "ccs_engine_kernel.cuh"

namespace ccs {

engine_fn engine_kernel_512_d7(int dmax) {
    return dmax == 7 ? k_engine<7, 512> : k_engine<8, 512>;
}

}  // namespace ccs

// ccs_engine_k512_d5_6.cu -- persistent engine kernel instances
// k_engine<5, 512> and k_engine<6, 512>.
#include "ccs_engine_kernel.cuh"

namespace ccs {

engine_fn engine_kernel_512_d5(int dmax) {
    return dmax == 5 ? k_engine<5, 512> : k_engine<6, 512>;
}

}  // namespace ccs

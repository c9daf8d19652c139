// ccs_engine_k1024_d7_8.cu -- persistent engine kernel instances
// k_engine<7, 1024> and k_engine<8, 1024>.
#include "ccs_engine_kernel.cuh"

namespace ccs {

engine_fn engine_kernel_1024_d7(int dmax) {
    return dmax == 7 ? k_engine<7, 1024> : k_engine<8, 1024>;
}

}  // namespace ccs

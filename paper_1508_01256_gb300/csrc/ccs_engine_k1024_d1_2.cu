// ccs_engine_k1024_d1_2.cu -- persistent engine kernel instances
// k_engine<1, 1024> and k_engine<2, 1024>.
#include "ccs_engine_kernel.cuh"

namespace ccs {

engine_fn engine_kernel_1024_d1(int dmax) {
    return dmax == 1 ? k_engine<1, 1024> : k_engine<2, 1024>;
}

}  // namespace ccs

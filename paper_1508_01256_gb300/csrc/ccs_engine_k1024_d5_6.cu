// ccs_engine_k1024_d5_6.cu -- persistent engine kernel instances
// k_engine<5, 1024> and k_engine<6, 1024>.
#include "ccs_engine_kernel.cuh"

namespace ccs {

engine_fn engine_kernel_1024_d5(int dmax) {
    return dmax == 5 ? k_engine<5, 1024> : k_engine<6, 1024>;
}

}  // namespace ccs

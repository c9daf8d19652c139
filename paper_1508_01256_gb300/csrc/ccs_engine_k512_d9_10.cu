// ccs_engine_k512_d9_10.cu -- persistent engine kernel instances
// k_engine<9, 512> and k_engine<10, 512>.
#include "ccs_engine_kernel.cuh"

namespace ccs {

engine_fn engine_kernel_512_d9(int dmax) {
    return dmax == 9 ? k_engine<9, 512> : k_engine<10, 512>;
}

}  // namespace ccs

// ccs_engine_k512_d13_14.cu -- persistent engine kernel instances
// k_engine<13, 512> and k_engine<14, 512>.
#include "ccs_engine_kernel.cuh"

namespace ccs {

engine_fn engine_kernel_512_d13(int dmax) {
    return dmax == 13 ? k_engine<13, 512> : k_engine<14, 512>;
}

}  // namespace ccs

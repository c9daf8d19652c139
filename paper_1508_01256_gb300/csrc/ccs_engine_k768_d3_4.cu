// ccs_engine_k768_d3_4.cu -- persistent engine kernel instances
// k_engine<3, 768> and k_engine<4, 768>.
#include "ccs_engine_kernel.cuh"

namespace ccs {

engine_fn engine_kernel_768_d3(int dmax) {
    return dmax == 3 ? k_engine<3, 768> : k_engine<4, 768>;
}

}  // namespace ccs

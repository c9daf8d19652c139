// ccs_engine_k768_d1_2.cu -- persistent engine kernel instances
// k_engine<1, 768> and k_engine<2, 768>.
#include "ccs_engine_kernel.cuh"

namespace ccs {

engine_fn engine_kernel_768_d1(int dmax) {
    return dmax == 1 ? k_engine<1, 768> : k_engine<2, 768>;
}

}  // namespace ccs

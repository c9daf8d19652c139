// ccs_engine_k768_d7_8.cu -- persistent engine kernel instances
// k_engine<7, 768> and k_engine<8, 768>.
#include "ccs_engine_kernel.cuh"

namespace ccs {

engine_fn engine_kernel_768_d7(int dmax) {
    return dmax == 7 ? k_engine<7, 768> : k_engine<8, 768>;
}

}  // namespace ccs

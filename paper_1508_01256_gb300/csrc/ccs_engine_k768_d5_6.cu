// ccs_engine_k768_d5_6.cu -- persistent engine kernel instances
// k_engine<5, 768> and k_engine<6, 768>.
#include "ccs_engine_kernel.cuh"

namespace ccs {

engine_fn engine_kernel_768_d5(int dmax) {
    return dmax == 5 ? k_engine<5, 768> : k_engine<6, 768>;
}

}  // namespace ccs

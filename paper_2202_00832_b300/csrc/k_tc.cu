// Mixed-precision (tcgen05) stages: placeholder until the tensor-core
// kernels land.
#include "common.cuh"

namespace loaf {

void run_energy_mixed(loaf_ctx* c, int W, int mode, int precision, const double2* theta,
                      double2* e_out, double2* e_pairs) {
    (void)c; (void)W; (void)mode; (void)precision; (void)theta; (void)e_out; (void)e_pairs;
    throw Error{LOAF_ERR_UNSUPPORTED, "mixed-precision path not built yet"};
}

void setup_mixed_operands(loaf_ctx* c, int mode, bool bf16) { (void)c; (void)mode; (void)bf16; }

}  // namespace loaf

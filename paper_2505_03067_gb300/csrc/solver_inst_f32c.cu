// solver_inst_f32c.cu -- solver kernel instances (the solve and the whole-step
// kernel of each), one translation unit per pair so the build runs in parallel.
#include "solver_kernels.cuh"

namespace mpm {

Variant inst_f32_8_1_1_1024() { return var_of<float, 8, 1, 1, 1024>(); }
Variant inst_f32_8_1_2_512() { return var_of<float, 8, 1, 2, 512>(); }

}  // namespace mpm

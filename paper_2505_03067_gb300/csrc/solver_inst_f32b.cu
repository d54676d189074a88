// solver_inst_f32b.cu -- solver kernel instances (the solve and the whole-step
// kernel of each), one translation unit per pair so the build runs in parallel.
#include "solver_kernels.cuh"

namespace mpm {

Variant inst_f32_8_2_2_512() { return var_of<float, 8, 2, 2, 512>(); }
Variant inst_f32_8_2_1_512() { return var_of<float, 8, 2, 1, 512>(); }

}  // namespace mpm

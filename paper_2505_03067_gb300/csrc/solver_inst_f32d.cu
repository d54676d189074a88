// solver_inst_f32d.cu -- solver kernel instances (the solve and the whole-step
// kernel of each), one translation unit per pair so the build runs in parallel.
#include "solver_kernels.cuh"

namespace mpm {

Variant inst_f32_8_1_1_640() { return var_of<float, 8, 1, 1, 640>(); }
Variant inst_f32_16_1_1_512() { return var_of<float, 16, 1, 1, 512>(); }

}  // namespace mpm

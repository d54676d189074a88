// solver_inst_f32e.cu -- solver kernel instances (the solve and the whole-step
// kernel of each), one translation unit per pair so the build runs in parallel.
#include "solver_kernels.cuh"

namespace mpm {

Variant inst_f32_32_1_1_512() { return var_of<float, 32, 1, 1, 512>(); }

}  // namespace mpm

// solver_inst_f64d.cu -- solver kernel instances (the solve and the whole-step
// kernel of each), one translation unit per pair so the build runs in parallel.
#include "solver_kernels.cuh"

namespace mpm {

Variant inst_f64_16_1_1_512() { return var_of<double, 16, 1, 1, 512>(); }
Variant inst_f64_32_1_1_512() { return var_of<double, 32, 1, 1, 512>(); }

}  // namespace mpm

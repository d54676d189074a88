// solver_inst_f64a.cu -- solver kernel instances (the solve and the whole-step
// kernel of each), one translation unit per pair so the build runs in parallel.
#include "solver_kernels.cuh"

namespace mpm {

Variant inst_f64_8_2_1_512() { return var_of<double, 8, 2, 1, 512>(); }
Variant inst_f64_8_1_2_512() { return var_of<double, 8, 1, 2, 512>(); }

}  // namespace mpm

// solver_inst_f64c.cu -- solver kernel instances (the solve and the whole-step
// kernel of each), one translation unit per pair so the build runs in parallel.
#include "solver_kernels.cuh"

namespace mpm {

Variant inst_f64_8_1_1_768() { return var_of<double, 8, 1, 1, 768>(); }
Variant inst_f64_8_2_1_768() { return var_of<double, 8, 2, 1, 768>(); }

}  // namespace mpm

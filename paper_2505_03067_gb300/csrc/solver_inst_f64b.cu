// solver_inst_f64b.cu -- solver kernel instances (the solve and the whole-step
// kernel of each), one translation unit per pair so the build runs in parallel.
#include "solver_kernels.cuh"

namespace mpm {

Variant inst_f64_8_1_1_512() { return var_of<double, 8, 1, 1, 512>(); }
Variant inst_f64_8_1_1_1024() { return var_of<double, 8, 1, 1, 1024>(); }

}  // namespace mpm

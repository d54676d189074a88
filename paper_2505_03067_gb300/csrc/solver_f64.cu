// solver_f64.cu -- instantiations of the FP64 solver kernels, restart <= 8,
// variants 0, 1 and 5.
#include "solver_kernels.cuh"

namespace mpm {

Variant pick_f64(int maxm, int variant)
{
    (void)maxm;
    switch (variant) {
    case 1: return var_of<double, 8, 1, 2, 512>();
    case 5: return var_of<double, 8, 1, 1, 512>();
    default: return var_of<double, 8, 2, 1, 512>();
    }
}

}  // namespace mpm

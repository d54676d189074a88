// solver_f64x.cu -- instantiations of the FP64 solver kernels: restart <= 8
// variants 2, 3 and 4, and the restart buckets 16 and 32.
#include "solver_kernels.cuh"

namespace mpm {

Variant pick_f64x(int maxm, int variant)
{
    if (maxm == 8) {
        switch (variant) {
        case 2: return var_of<double, 8, 1, 1, 1024>();
        case 3: return var_of<double, 8, 1, 1, 768>();
        default: return var_of<double, 8, 2, 1, 768>();
        }
    }
    if (maxm == 16) return var_of<double, 16, 1, 1, 512>();
    return var_of<double, 32, 1, 1, 512>();
}

}  // namespace mpm

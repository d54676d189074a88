// solver_f32.cu -- instantiations of the FP32-basis solver kernels (the
// solve and the whole-step kernel of every variant).
#include "solver_kernels.cuh"

namespace mpm {

Variant pick_f32(int maxm, int variant)
{
    if (maxm == 8) {
        switch (variant) {
        case 1: return var_of<float, 8, 1, 1, 768>();
        case 2: return var_of<float, 8, 2, 2, 512>();
        case 3: return var_of<float, 8, 2, 1, 512>();
        case 4: return var_of<float, 8, 1, 1, 1024>();
        case 5: return var_of<float, 8, 1, 2, 512>();
        case 6: return var_of<float, 8, 1, 1, 640>();
        default: return var_of<float, 8, 1, 1, 512>();
        }
    }
    if (maxm == 16) return var_of<float, 16, 1, 1, 512>();
    return var_of<float, 32, 1, 1, 512>();
}

}  // namespace mpm

// Instances of the register-staged scan kernel (8-bit symbols) with the
// prefix bitmap as the first stage and the prefix entries read through L2
// (one translation unit per group, so that they compile in parallel).
#include "kernels_r.cuh"

namespace pfac {

void *scan_kernel_r8_g0_f(int rep) {
    switch (rep) {
        case 0: return (void *)k_scanr<8, 0, 0, VAR_F>;
        case 1: return (void *)k_scanr<8, 1, 0, VAR_F>;
        case 2: return (void *)k_scanr<8, 2, 0, VAR_F>;
        case 3: return (void *)k_scanr<8, 3, 0, VAR_F>;
        case 4: return (void *)k_scanr<8, 4, 0, VAR_F>;
        default: return nullptr;
    }
}

}  // namespace pfac

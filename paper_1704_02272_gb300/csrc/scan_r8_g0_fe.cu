// Instances of the register-staged scan kernel (8-bit symbols) with the
// prefix bitmap as the first stage and the prefix entries in shared memory
// (one translation unit per group, so that they compile in parallel).
#include "kernels_r.cuh"

namespace pfac {

void *scan_kernel_r8_g0_fe(int rep) {
    switch (rep) {
        case 0: return (void *)k_scanr<8, 0, 0, VAR_FE>;
        case 1: return (void *)k_scanr<8, 1, 0, VAR_FE>;
        case 2: return (void *)k_scanr<8, 2, 0, VAR_FE>;
        case 3: return (void *)k_scanr<8, 3, 0, VAR_FE>;
        case 4: return (void *)k_scanr<8, 4, 0, VAR_FE>;
        default: return nullptr;
    }
}

}  // namespace pfac

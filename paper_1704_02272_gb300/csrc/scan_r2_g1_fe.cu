// Instances of the register-staged scan kernel (2-bit symbols) with the
// gram filter as the first stage and the prefix entries in shared memory
// (one translation unit per group, so that they compile in parallel).
#include "kernels_r.cuh"

namespace pfac {

template <int NW>
static void *pick(int rep) {
    switch (rep) {
        case 0: return (void *)k_scanr<2, 0, 0, 1, VAR_FE, NW>;
        case 1: return (void *)k_scanr<2, 0, 1, 1, VAR_FE, NW>;
        case 2: return (void *)k_scanr<2, 0, 2, 1, VAR_FE, NW>;
        case 3: return (void *)k_scanr<2, 0, 3, 1, VAR_FE, NW>;
        case 4: return (void *)k_scanr<2, 0, 4, 1, VAR_FE, NW>;
        default: return nullptr;
    }
}

void *scan_kernel_r2_g1_fe(int rep, int nw) {
    if (nw == RNW) return pick<RNW>(rep);
    if (nw == RNW_WIDE) return pick<RNW_WIDE>(rep);
    return nullptr;
}

}  // namespace pfac

// Instances of the register-staged scan kernel (2-bit symbols) over the dense
// layout's transition table (record format 3), gram filter as the first
// stage, default CTA width: the uncompressed table in the same kernel as the
// compressed one.
#include "kernels_r.cuh"

namespace pfac {

template <int VAR>
static void *pick(int rep) {
    switch (rep) {
        case 0: return (void *)k_scanr<2, 3, 0, 1, VAR, RNW>;
        case 1: return (void *)k_scanr<2, 3, 1, 1, VAR, RNW>;
        case 2: return (void *)k_scanr<2, 3, 2, 1, VAR, RNW>;
        case 3: return (void *)k_scanr<2, 3, 3, 1, VAR, RNW>;
        case 4: return (void *)k_scanr<2, 3, 4, 1, VAR, RNW>;
        default: return nullptr;
    }
}

void *scan_kernel_r2_d1(int rep, int var, int nw) {
    if (nw != RNW) return nullptr;
    return var == VAR_FE ? pick<VAR_FE>(rep) : pick<VAR_F>(rep);
}

}  // namespace pfac

// Instances of the resolver kernel, one per record format.
#include "kernels_r.cuh"

namespace pfac {

void *resolve_kernel(int w) {
    switch (w) {
        case 0: return (void *)k_resolve<0>;
        case 1: return (void *)k_resolve<1>;
        case 2: return (void *)k_resolve<2>;
        case 3: return (void *)k_resolve<3>;
        case 8: return (void *)k_resolve<8>;
        default: return nullptr;
    }
}

}  // namespace pfac

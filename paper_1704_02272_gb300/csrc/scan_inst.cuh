// Instantiates the queued scan kernel for one symbol width PFAC_SCAN_BPS
// and exports a lookup of its entry points (one translation unit per width
// keeps compile times parallel).
#include "kernels_q.cuh"

#define PFAC_CAT2(a, b) a##b
#define PFAC_CAT(a, b) PFAC_CAT2(a, b)

namespace pfac {

static constexpr int kBps = PFAC_SCAN_BPS;
static constexpr int kW = kBps <= 5 ? 1 : (kBps == 6 ? 2 : 8);

void *PFAC_CAT(scan_kernel_bps, PFAC_SCAN_BPS)(int var, int emit) {
    switch (var * 2 + (emit ? 1 : 0)) {
        case VAR_F * 2: return (void *)k_scanq<kW, kBps, VAR_F, 0>;
        case VAR_F * 2 + 1: return (void *)k_scanq<kW, kBps, VAR_F, 1>;
        case VAR_FE * 2: return (void *)k_scanq<kW, kBps, VAR_FE, 0>;
        case VAR_FE * 2 + 1: return (void *)k_scanq<kW, kBps, VAR_FE, 1>;
        default: return nullptr;
    }
}

}  // namespace pfac

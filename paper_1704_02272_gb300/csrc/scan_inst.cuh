// Instantiates the scan kernel variants for one symbol width PFAC_SCAN_BPS
// and exports a lookup of their entry points (one translation unit per
// width keeps compile times parallel).
#include "kernels.cuh"

#define PFAC_CAT2(a, b) a##b
#define PFAC_CAT(a, b) PFAC_CAT2(a, b)

namespace pfac {

static constexpr int kBps = PFAC_SCAN_BPS;
static constexpr int kW = kBps <= 5 ? 1 : (kBps == 6 ? 2 : 8);

void *PFAC_CAT(scan_kernel_bps, PFAC_SCAN_BPS)(int var) {
    switch (var) {
        case VAR_FILTER: return (void *)k_scan<kW, kBps, VAR_FILTER>;
        case VAR_DSMEM: return (void *)k_scan<kW, kBps, VAR_DSMEM>;
        case VAR_DGLOBAL: return (void *)k_scan<kW, kBps, VAR_DGLOBAL>;
        default: return nullptr;
    }
}

}  // namespace pfac

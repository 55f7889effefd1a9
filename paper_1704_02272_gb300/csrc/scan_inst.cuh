// Instantiates the queued scan kernel for one symbol width PFAC_SCAN_BPS
// and exports a lookup of its entry points (one translation unit per width
// keeps compile times parallel).  Alphabets of up to 8 symbols have two
// record formats: packed (W = 0) in every configuration, and the two-word
// records of the 32-symbol format (W = 1, tries too large to pack, or built
// with wide records) for the default CTA width.  Rows of the dense layout's
// transition table (W = 3) run in the same kernel, default CTA width.
#include "kernels_q.cuh"

#define PFAC_CAT2(a, b) a##b
#define PFAC_CAT(a, b) PFAC_CAT2(a, b)

namespace pfac {

static constexpr int kBps = PFAC_SCAN_BPS;
static constexpr int kW = kBps <= 3 ? 0 : (kBps <= 5 ? 1 : (kBps == 6 ? 2 : 8));

template <int W, int NW>
static void *scan_kernel_nw(int var, int emit) {
    switch (var * 2 + (emit ? 1 : 0)) {
        case VAR_F * 2: return (void *)k_scanq<W, kBps, VAR_F, 0, NW>;
        case VAR_F * 2 + 1: return (void *)k_scanq<W, kBps, VAR_F, 1, NW>;
        case VAR_FE * 2: return (void *)k_scanq<W, kBps, VAR_FE, 0, NW>;
        case VAR_FE * 2 + 1: return (void *)k_scanq<W, kBps, VAR_FE, 1, NW>;
        default: return nullptr;
    }
}

void *PFAC_CAT(scan_kernel_bps, PFAC_SCAN_BPS)(int var, int emit, int nw, int w) {
    if (var == (VAR_F | VAR_MERGED)) {  // merged tries: one configuration
        if (w != kW || nw != QW) return nullptr;
        return emit ? (void *)k_scanq<kW, kBps, VAR_F | VAR_MERGED, 1, QW>
                    : (void *)k_scanq<kW, kBps, VAR_F | VAR_MERGED, 0, QW>;
    }
    if (w == kW) {
        if (nw == QW) return scan_kernel_nw<kW, QW>(var, emit);
        if (nw == QW_WIDE) return scan_kernel_nw<kW, QW_WIDE>(var, emit);
        return nullptr;
    }
    if (kW == 0 && w == 1 && nw == QW) return scan_kernel_nw<kW == 0 ? 1 : kW, QW>(var, emit);
    // the dense layout's transition table in the same kernel
    if (w == 3 && nw == QW) return scan_kernel_nw<3, QW>(var, emit);
    return nullptr;
}

}  // namespace pfac

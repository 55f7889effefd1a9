// Scan-kernel instances for prefix indices of 6 bits per symbol.
#define PFAC_SCAN_BPS 6
#include "scan_inst.cuh"

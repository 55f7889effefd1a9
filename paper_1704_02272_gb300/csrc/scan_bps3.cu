// Scan-kernel instances for prefix indices of 3 bits per symbol.
#define PFAC_SCAN_BPS 3
#include "scan_inst.cuh"

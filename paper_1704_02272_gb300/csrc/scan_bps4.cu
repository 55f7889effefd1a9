// Scan-kernel instances for prefix indices of 4 bits per symbol.
#define PFAC_SCAN_BPS 4
#include "scan_inst.cuh"

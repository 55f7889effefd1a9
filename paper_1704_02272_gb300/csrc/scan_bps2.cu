// Scan-kernel instances for prefix indices of 2 bits per symbol.
#define PFAC_SCAN_BPS 2
#include "scan_inst.cuh"

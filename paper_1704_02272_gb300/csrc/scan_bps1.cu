// Scan-kernel instances for prefix indices of 1 bits per symbol.
#define PFAC_SCAN_BPS 1
#include "scan_inst.cuh"

// Scan-kernel instances for prefix indices of 8 bits per symbol.
#define PFAC_SCAN_BPS 8
#include "scan_inst.cuh"

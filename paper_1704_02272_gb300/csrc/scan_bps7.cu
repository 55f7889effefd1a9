// Scan-kernel instances for prefix indices of 7 bits per symbol.
#define PFAC_SCAN_BPS 7
#include "scan_inst.cuh"

// Scan-kernel instances for prefix indices of 5 bits per symbol.
#define PFAC_SCAN_BPS 5
#include "scan_inst.cuh"

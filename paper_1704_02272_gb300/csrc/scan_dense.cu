// Scan-kernel instance for the uncompressed state-transition table.
#include "kernels.cuh"

namespace pfac {

void *scan_kernel_dense() { return (void *)k_scan<1, 8, VAR_DENSE>; }

}  // namespace pfac

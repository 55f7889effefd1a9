// Scan-kernel instance for the uncompressed state-transition table.
#define PFAC_DEFINE_DENSE_KERNEL
#include "kernels.cuh"

namespace pfac {

void *scan_kernel_dense() { return (void *)k_scan_dense; }

}  // namespace pfac

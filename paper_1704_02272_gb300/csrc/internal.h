// Host-side table object and error reporting shared by the library's
// translation units.
#pragma once
#include <stdarg.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "../../include/pfac.h"
#include "table.h"

struct pfac_table {
    pfac::DevTable dev;
    void *d_blob = nullptr;
    uint64_t blob_bytes = 0;
    // host-only tables keep their blob here (the DevTable's pointers point
    // into it; no kernel reads them: every match call refuses such a table)
    std::vector<uint8_t> h_blob;
    pfac_table_info_t info{};
    uint32_t kmin = 0, kmax = 0;  // prefix nodes exist for depths kmin..kmax
    int device = 0;
    // autotuned defaults (0 = none)
    uint32_t tuned_variant = 0;
    uint32_t tuned_k = 0;
    uint32_t tuned_copies = 0;
    uint32_t tuned_masks = 0;
    uint32_t tuned_gram = 0;
    uint32_t tuned_bytes = 0;
    uint32_t tuned_nw = 0;
    uint32_t tuned_kernel = 0;
    uint32_t tuned_records = 0;
    uint32_t tuned_resolver = 0;
    double match_density = 0.0;  // expected matches per position of uniform text
};

namespace pfac {

int set_error(int status, const char *fmt, ...);
void clear_error();

// PFAC_OK when the current device and, for a non-NULL stream, the stream's
// device are the device the table was uploaded to; otherwise PFAC_EINVAL
// (with a message naming `who`), so that no kernel is launched on one GPU
// with another GPU's pointers.
int check_table_device(const pfac_table *t, void *cuda_stream, const char *who);

}  // namespace pfac

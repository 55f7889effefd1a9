// pfac_match_noalloc: the matching pipeline with its scratch memory taken
// from a fixed array compiled into the library instead of a caller- or
// library-allocated workspace.
//
// Some callers cannot allocate device memory at the moment they need to
// match: code running inside a custom allocator's callback, a host-side
// real-time loop that must not take the allocator's locks or risk an
// out-of-memory failure mid-stream, or a host function in a process whose
// memory budget is fixed after start-up.  For them this entry point performs
// no cudaMalloc, no cudaFree and no call into an allocating library: the
// scratch (per-tile counters, match records and segment lists) lives in
// `g_noalloc_scratch` below, a file-scope device array of
// PFAC_NOALLOC_SCRATCH_BYTES that every GPU which loads this library holds
// until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

static __device__ __align__(256) uint8_t g_noalloc_scratch[PFAC_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of this device's copy of the array.  In host code the
// array's name is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress, once per device, with that device current.
int scratch_for_current_device(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return pfac::set_error(PFAC_ECUDA, "pfac_match_noalloc: cudaGetDevice: %s",
                               cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return pfac::set_error(PFAC_EINVAL, "pfac_match_noalloc: device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return pfac::set_error(PFAC_ECUDA, "pfac_match_noalloc: cudaGetSymbolAddress: %s",
                                   cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return PFAC_OK;
}

}  // namespace

extern "C" int pfac_match_noalloc(const pfac_table *t, const uint8_t *d_input, uint64_t n_bytes,
                                  const uint64_t *d_seg_offsets, uint32_t n_segments,
                                  uint64_t *d_out_keys, uint64_t out_capacity, uint64_t *d_count,
                                  int32_t *d_status, const pfac_match_opts *opts,
                                  void *cuda_stream) {
    pfac::clear_error();
    if (!t) return pfac::set_error(PFAC_EINVAL, "pfac_match_noalloc: NULL table");
    uint64_t need = 0;
    int rc = pfac_workspace_bytes(t, n_bytes, n_segments, opts, &need);
    if (rc) return rc;
    if (need > (uint64_t)PFAC_NOALLOC_SCRATCH_BYTES)
        return pfac::set_error(PFAC_EINVAL,
                               "pfac_match_noalloc: an input of %llu bytes in %u segments needs "
                               "%llu bytes of scratch, more than the built-in %llu; split the "
                               "input or use pfac_match_async with a workspace",
                               (unsigned long long)n_bytes, n_segments,
                               (unsigned long long)need,
                               (unsigned long long)PFAC_NOALLOC_SCRATCH_BYTES);
    void *scratch = nullptr;
    rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    // The shared array keeps whatever the previous call left in it; the
    // pipeline clears the part that must start at zero (its header) on the
    // stream before the first kernel, and writes every other part before it
    // reads it.
    return pfac_match_async(t, d_input, n_bytes, d_seg_offsets, n_segments, d_out_keys,
                            out_capacity, d_count, d_status, scratch, need, opts, cuda_stream);
}

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
#include <string.h>

#include <mutex>

#include "internal.h"

static __device__ __align__(256) uint8_t g_noalloc_scratch[PFAC_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
// Per device: the CUDA context the address was looked up in, and the
// address.  A device whose context was destroyed and created again (a
// cudaDeviceReset) gets a new lookup when its current context differs.
struct ScratchAddr {
    void *ctx = nullptr;
    void *ptr = nullptr;
};
ScratchAddr g_scratch[kMaxDevices];

// The driver's cuCtxGetCurrent, reached through the runtime so the library
// needs no link against the driver library; nullptr when unavailable.
typedef int (*CtxGetCurrentFn)(void **);
CtxGetCurrentFn ctx_get_current() {
    static CtxGetCurrentFn fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            f = nullptr;
        }
        return (CtxGetCurrentFn)f;
    }();
    return fn;
}

void *current_context() {
    void *ctx = nullptr;
    CtxGetCurrentFn f = ctx_get_current();
    if (!f || f(&ctx) != 0) return nullptr;
    return ctx;
}

// Device address of this device's copy of the array.  In host code the
// array's name is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress with the device current; it is looked up on the first
// call on a device (and again after that device's context was replaced).
int scratch_for_current_device(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return pfac::set_error(PFAC_ECUDA, "pfac_match_noalloc: cudaGetDevice: %s",
                               cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return pfac::set_error(PFAC_EINVAL, "pfac_match_noalloc: device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    ScratchAddr &c = g_scratch[dev];
    void *ctx = current_context();
    if (!c.ptr || !ctx || c.ctx != ctx) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return pfac::set_error(PFAC_ECUDA, "pfac_match_noalloc: cudaGetSymbolAddress: %s",
                                   cudaGetErrorString(e));
        }
        c.ptr = p;
        c.ctx = current_context();  // the runtime's context exists now
    }
    *out = c.ptr;
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
    if (!t->d_blob)
        return pfac::set_error(PFAC_EINVAL, "pfac_match_noalloc: table was built host-only");
    int rc = pfac::check_table_device(t, cuda_stream, "pfac_match_noalloc");
    if (rc) return rc;
    uint64_t need = 0;
    rc = pfac_workspace_bytes(t, n_bytes, n_segments, opts, &need);
    if (rc) return rc;
    // library choices that take more scratch (a record per position, 8 bytes
    // per input byte; the resolver kernel's buffer) give way to the smaller
    // record space and the scan's own resolution when only those fit
    pfac_match_opts o32;
    if (need > (uint64_t)PFAC_NOALLOC_SCRATCH_BYTES &&
        !(opts && opts->records_per_slice && opts->resolver)) {
        if (opts) o32 = *opts;
        else memset(&o32, 0, sizeof o32);
        if (!o32.records_per_slice) o32.records_per_slice = 32;
        if (!o32.resolver) o32.resolver = 1;
        uint64_t need32 = 0;
        if (pfac_workspace_bytes(t, n_bytes, n_segments, &o32, &need32) == PFAC_OK &&
            need32 <= (uint64_t)PFAC_NOALLOC_SCRATCH_BYTES) {
            opts = &o32;
            need = need32;
        }
        pfac::clear_error();
    }
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

// pfac_match_host: matching of a text in host memory with the host-device
// copies pipelined against the matching.  The text is cut into chunks of
// start positions; chunk i is matched on the caller's stream over its bytes
// plus a read halo of max_len - 1 (starts_end / position_base keep its keys
// to its own starts, in global positions), while later chunks are copied in
// on one library stream and earlier chunks' keys are copied out on another.
// Three slots of device buffers rotate.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "internal.h"

using namespace pfac;

namespace {

// Pinned staging for the chunks' local segment offsets, kept between calls
// (allocating pinned memory per call costs more than the copies it serves).
std::mutex g_host_mu;
constexpr int NSLOT = 3;  // chunks in flight: copy in, match, copy out
uint64_t *g_pin[NSLOT] = {nullptr, nullptr, nullptr};
size_t g_pin_words[NSLOT] = {0, 0, 0};
uint64_t *g_pin_small = nullptr;  // per slot: count, status

bool pin_reserve(int s, size_t words) {
    if (g_pin_words[s] >= words) return true;
    if (g_pin[s]) cudaFreeHost(g_pin[s]);
    g_pin[s] = nullptr;
    g_pin_words[s] = 0;
    if (cudaHostAlloc((void **)&g_pin[s], words * 8, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    g_pin_words[s] = words;
    return true;
}

struct Slot {
    uint8_t *in = nullptr;      // chunk text
    uint64_t *seg = nullptr;    // chunk's local segment offsets
    void *ws = nullptr;         // workspace
    uint64_t *keys = nullptr;   // chunk keys
    uint64_t *small = nullptr;  // count (8 B) and status (4 B)
    cudaEvent_t h2d = nullptr, done = nullptr, d2h = nullptr;
};

// Streams, events and device buffers of one device, kept between calls and
// grown on demand (mapping fresh device memory per call costs milliseconds).
struct HostCtx {
    bool init = false;
    cudaStream_t h2d = nullptr, d2h = nullptr;
    Slot sl[NSLOT];
    uint64_t in_cap = 0, seg_cap = 0, ws_cap = 0, keys_cap = 0;
    uint64_t keys_hint = 0;  // largest chunk key count seen (keys)
};
constexpr int MAX_DEV = 64;
HostCtx g_ctx[MAX_DEV];

cudaError_t grow(void **p, uint64_t &cap, uint64_t want) {
    if (cap >= want && *p) return cudaSuccess;
    if (*p) cudaFree(*p);
    *p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(p, want);
    if (e == cudaSuccess) cap = want;
    return e;
}

cudaError_t ctx_prepare(HostCtx &c, uint64_t in_b, uint64_t seg_b, uint64_t ws_b,
                        uint64_t keys_b) {
    cudaError_t e = cudaSuccess;
    if (!c.init) {
        e = cudaStreamCreateWithFlags(&c.h2d, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c.d2h, cudaStreamNonBlocking);
        for (int s = 0; s < NSLOT && e == cudaSuccess; s++) {
            e = cudaEventCreateWithFlags(&c.sl[s].h2d, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.sl[s].done, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.sl[s].d2h, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaMalloc((void **)&c.sl[s].small, 16);
        }
        if (e != cudaSuccess) return e;
        c.init = true;
    }
    // every slot is sized alike, so one capacity per buffer kind
    uint64_t cap[4];
    const uint64_t want[4] = {in_b, seg_b, ws_b, keys_b};
    const uint64_t have[4] = {c.in_cap, c.seg_cap, c.ws_cap, c.keys_cap};
    for (int s = 0; s < NSLOT && e == cudaSuccess; s++) {
        void **bufs[4] = {(void **)&c.sl[s].in, (void **)&c.sl[s].seg, &c.sl[s].ws,
                          (void **)&c.sl[s].keys};
        for (int b = 0; b < 4 && e == cudaSuccess; b++) {
            cap[b] = have[b];
            e = grow(bufs[b], cap[b], std::max(want[b], have[b]));
        }
    }
    if (e == cudaSuccess) {
        c.in_cap = cap[0];
        c.seg_cap = cap[1];
        c.ws_cap = cap[2];
        c.keys_cap = cap[3];
    }
    return e;
}

}  // namespace

extern "C" void pfac_match_host_release(void) {
    std::lock_guard<std::mutex> lk(g_host_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) return;
    HostCtx &c = g_ctx[dev];
    if (!c.init) return;
    cudaDeviceSynchronize();
    for (int s = 0; s < NSLOT; s++) {
        cudaFree(c.sl[s].in);
        cudaFree(c.sl[s].seg);
        cudaFree(c.sl[s].ws);
        cudaFree(c.sl[s].keys);
        cudaFree(c.sl[s].small);
        cudaEventDestroy(c.sl[s].h2d);
        cudaEventDestroy(c.sl[s].done);
        cudaEventDestroy(c.sl[s].d2h);
    }
    cudaStreamDestroy(c.h2d);
    cudaStreamDestroy(c.d2h);
    c = HostCtx();
}

extern "C" int pfac_match_host(const pfac_table *t, const uint8_t *h_input, uint64_t n_bytes,
                               const uint64_t *h_seg, uint32_t n_segments, uint64_t *h_out_keys,
                               uint64_t out_capacity, uint64_t *n_out, uint64_t chunk_bytes,
                               const pfac_match_opts *opts, void *cuda_stream) {
    clear_error();
    if (!t || !n_out || (n_bytes && !h_input) || !h_seg)
        return set_error(PFAC_EINVAL, "pfac_match_host: NULL argument");
    if (!t->d_blob) return set_error(PFAC_EINVAL, "pfac_match_host: table was built host-only");
    {
        const int drc = check_table_device(t, cuda_stream, "pfac_match_host");
        if (drc) return drc;
    }
    if (out_capacity && !h_out_keys) return set_error(PFAC_EINVAL, "pfac_match_host: NULL output");
    if (opts && (opts->starts_end || opts->position_base))
        return set_error(PFAC_EINVAL, "pfac_match_host: starts_end and position_base are set "
                         "per chunk by the call");
    if (n_bytes >> (64 - PFAC_ID_BITS))
        return set_error(PFAC_EINVAL, "pfac_match_host: input longer than 2^%d bytes",
                         64 - PFAC_ID_BITS);
    if (n_bytes && n_segments == 0)
        return set_error(PFAC_EINVAL, "pfac_match_host: a non-empty input needs a segment");
    // segment offsets: 0 first, n_bytes last, non-decreasing
    if (h_seg[0] != 0 || h_seg[n_segments] != n_bytes)
        return set_error(PFAC_EINVAL, "pfac_match_host: offsets must run from 0 to n_bytes");
    for (uint32_t i = 0; i < n_segments; i++)
        if (h_seg[i + 1] < h_seg[i])
            return set_error(PFAC_EINVAL, "pfac_match_host: offsets decrease at %u", i);
    *n_out = 0;
    if (n_bytes == 0) return PFAC_OK;

    const uint64_t C = chunk_bytes ? ((chunk_bytes + 255) & ~255ull) : (32ull << 20);
    const uint64_t H = t->info.max_len ? t->info.max_len - 1 : 0;
    const uint64_t n_chunks = (n_bytes + C - 1) / C;
    const uint64_t *seg_end = h_seg + n_segments + 1;
    // chunk j: starts [a, b), bytes [a, e); local offsets: 0, the offsets
    // strictly inside (a, e), e - a
    auto bounds = [&](uint64_t j, uint64_t &a, uint64_t &b, uint64_t &e, const uint64_t *&lo,
                      const uint64_t *&hi) {
        a = j * C;
        b = std::min(a + C, n_bytes);
        e = std::min(b + H, n_bytes);
        lo = std::upper_bound(h_seg, seg_end, a);
        hi = std::lower_bound(lo, seg_end, e);
    };
    size_t max_local = 2;
    for (uint64_t j = 0; j < n_chunks; j++) {
        uint64_t a, b, e;
        const uint64_t *lo, *hi;
        bounds(j, a, b, e, lo, hi);
        max_local = std::max(max_local, (size_t)(hi - lo) + 2);
    }
    pfac_match_opts o;
    if (opts) o = *opts;
    else memset(&o, 0, sizeof o);
    uint64_t ws_bytes = 0;
    int rc = pfac_workspace_bytes(t, C + H, (uint32_t)(max_local - 1), &o, &ws_bytes);
    if (rc) return rc;

    std::lock_guard<std::mutex> lk(g_host_mu);
    if (!g_pin_small && cudaHostAlloc((void **)&g_pin_small, 64, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        g_pin_small = nullptr;
    }
    if (!g_pin_small || !pin_reserve(0, max_local) || !pin_reserve(1, max_local) ||
        !pin_reserve(2, max_local))
        return set_error(PFAC_ENOMEM, "pfac_match_host: pinned staging of %zu offsets", max_local);

    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess || dev < 0 || dev >= MAX_DEV)
        return set_error(PFAC_ECUDA, "pfac_match_host: no usable device");
    HostCtx &cx = g_ctx[dev];
    // keys per chunk held on the device (at least the most an earlier call
    // met, up to 2^28); a chunk with more is matched again alone afterwards
    const uint64_t hint = std::min<uint64_t>(cx.keys_hint, 1ull << 28);
    const uint64_t K = std::max<uint64_t>(std::max<uint64_t>(1ull << 20, C / 4), hint);
    ce = ctx_prepare(cx, C + H + 16, max_local * 8, ws_bytes, K * 8);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return set_error(ce == cudaErrorMemoryAllocation ? PFAC_ENOMEM : PFAC_ECUDA,
                         "pfac_match_host: device buffers: %s", cudaGetErrorString(ce));
    }
    cudaStream_t comp = (cudaStream_t)cuda_stream, h2d = cx.h2d, d2h = cx.d2h;
    Slot *sl = cx.sl;
    // the caller's stream may have work the chunks depend on (the table)
    cudaEvent_t ready = sl[0].h2d;
    ce = cudaEventRecord(ready, comp);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(h2d, ready, 0);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(d2h, ready, 0);

    struct Redo {
        uint64_t chunk, off, count;
    };
    std::vector<Redo> redo;
    uint64_t *hcnt[NSLOT] = {g_pin_small, g_pin_small + 2, g_pin_small + 4};  // count, status
    uint64_t total = 0;
    int status = PFAC_OK;

    // copies out the keys of chunk j once its count is known
    auto finish = [&](uint64_t j) -> bool {
        const int s = (int)(j % NSLOT);
        if (cudaEventSynchronize(sl[s].done) != cudaSuccess) return false;
        const uint64_t c = hcnt[s][0];
        const int32_t st = (int32_t)(uint32_t)hcnt[s][1];
        if (st != PFAC_OK && status == PFAC_OK) status = st;
        if (c > K) {
            redo.push_back({j, total, c});
            cx.keys_hint = std::max(cx.keys_hint, c + c / 8);
        } else if (total < out_capacity && c) {
            const uint64_t m = std::min(c, out_capacity - total);
            if (cudaMemcpyAsync(h_out_keys + total, sl[s].keys, m * 8, cudaMemcpyDeviceToHost,
                                d2h) != cudaSuccess)
                return false;
        }
        if (cudaEventRecord(sl[s].d2h, d2h) != cudaSuccess) return false;
        total += c;
        return true;
    };

    for (uint64_t i = 0; i < n_chunks && ce == cudaSuccess && rc == PFAC_OK; i++) {
        const int s = (int)(i % NSLOT);
        uint64_t a, b, e;
        const uint64_t *lo, *hi;
        bounds(i, a, b, e, lo, hi);
        // the slot's staging is free once the copies of chunk i - 2 are done
        if (i >= NSLOT) ce = cudaEventSynchronize(sl[s].h2d);
        if (ce != cudaSuccess) break;
        uint64_t *loc = g_pin[s];
        size_t nl = 0;
        loc[nl++] = 0;
        for (const uint64_t *p = lo; p < hi; p++) loc[nl++] = *p - a;
        loc[nl++] = e - a;
        if (i >= NSLOT) ce = cudaStreamWaitEvent(h2d, sl[s].done, 0);  // chunk i - 3 read its input
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(sl[s].in, h_input + a, e - a, cudaMemcpyHostToDevice, h2d);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(sl[s].seg, loc, nl * 8, cudaMemcpyHostToDevice, h2d);
        if (ce == cudaSuccess) ce = cudaEventRecord(sl[s].h2d, h2d);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(comp, sl[s].h2d, 0);
        if (ce == cudaSuccess && i >= NSLOT) ce = cudaStreamWaitEvent(comp, sl[s].d2h, 0);
        if (ce != cudaSuccess) break;
        o.starts_end = b - a;
        o.position_base = a;
        rc = pfac_match_async(t, sl[s].in, e - a, sl[s].seg, (uint32_t)(nl - 1), sl[s].keys, K,
                              sl[s].small, (int32_t *)(sl[s].small + 1), sl[s].ws, ws_bytes, &o,
                              comp);
        if (rc != PFAC_OK) break;
        ce = cudaMemcpyAsync(hcnt[s], sl[s].small, 16, cudaMemcpyDeviceToHost, comp);
        if (ce == cudaSuccess) ce = cudaEventRecord(sl[s].done, comp);
        // the host waits for the oldest chunk in flight, two behind
        if (ce == cudaSuccess && i >= NSLOT - 1 && !finish(i - (NSLOT - 1))) ce = cudaErrorUnknown;
    }
    for (uint64_t j = n_chunks > NSLOT - 1 ? n_chunks - (NSLOT - 1) : 0;
         j < n_chunks && ce == cudaSuccess && rc == PFAC_OK; j++)
        if (!finish(j)) ce = cudaErrorUnknown;
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(d2h);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(h2d);

    // chunks with more keys than a slot holds, one at a time
    for (const Redo &r : redo) {
        if (ce != cudaSuccess || rc != PFAC_OK) break;
        if (r.off >= out_capacity) continue;
        uint64_t a, b, e;
        const uint64_t *lo, *hi;
        bounds(r.chunk, a, b, e, lo, hi);
        uint64_t *loc = g_pin[0];
        size_t nl = 0;
        loc[nl++] = 0;
        for (const uint64_t *p = lo; p < hi; p++) loc[nl++] = *p - a;
        loc[nl++] = e - a;
        uint64_t *big = nullptr;
        ce = cudaMallocAsync((void **)&big, r.count * 8, comp);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(sl[0].in, h_input + a, e - a, cudaMemcpyHostToDevice, comp);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(sl[0].seg, loc, nl * 8, cudaMemcpyHostToDevice, comp);
        if (ce == cudaSuccess) {
            o.starts_end = b - a;
            o.position_base = a;
            rc = pfac_match_async(t, sl[0].in, e - a, sl[0].seg, (uint32_t)(nl - 1), big, r.count,
                                  sl[0].small, (int32_t *)(sl[0].small + 1), sl[0].ws, ws_bytes,
                                  &o, comp);
        }
        if (ce == cudaSuccess && rc == PFAC_OK) {
            const uint64_t m = std::min(r.count, out_capacity - r.off);
            ce = cudaMemcpyAsync(h_out_keys + r.off, big, m * 8, cudaMemcpyDeviceToHost, comp);
        }
        if (big) cudaFreeAsync(big, comp);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(comp);
    }

    // the buffers stay for the next call; wait until every stream drained
    cudaError_t ce2 = cudaStreamSynchronize(comp);
    if (ce2 == cudaSuccess) ce2 = cudaStreamSynchronize(h2d);
    if (ce2 == cudaSuccess) ce2 = cudaStreamSynchronize(d2h);
    if (rc != PFAC_OK) return rc;
    if (ce == cudaSuccess) ce = ce2;
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return set_error(PFAC_ECUDA, "pfac_match_host: %s", cudaGetErrorString(ce));
    }
    if (status != PFAC_OK) return set_error(status, "pfac_match_host: device reported %d", status);
    *n_out = total;
    if (total > out_capacity)
        return set_error(PFAC_ENOSPC, "pfac_match_host: %llu keys, room for %llu",
                         (unsigned long long)total, (unsigned long long)out_capacity);
    return PFAC_OK;
}

// pfac_verify: the secondary process of prefix matching (Section 2.4).  A
// table built with truncate_depth d reports every (p, j) whose first
// min(|P_j|, d) symbols occur at p; this keeps those whose whole pattern
// occurs there inside p's segment, in key order.  Three kernels: mark (one
// thread per candidate compares the pattern's tail and counts the kept ones
// per tile), scan (one CTA turns the tile counts into offsets and the
// total), compact (each tile writes its kept keys at its offset, in order).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "internal.h"

using namespace pfac;

namespace {

constexpr int VT = 1024;  // candidates per tile = threads per CTA

struct VerifyParams {
    const uint8_t *in;
    uint64_t n;
    const uint64_t *seg;
    uint32_t n_seg;
    const uint64_t *keys;
    uint64_t n_keys;
    uint64_t *out;
    uint64_t *count;
    uint8_t *flag;       // per candidate: kept
    uint64_t *tile_cnt;  // per tile: kept, then the tile's output offset
    uint64_t n_tiles;
    const uint8_t *pat;
    const uint32_t *pat_off;
    uint32_t n_pat;
    uint32_t trunc;
};

__device__ __forceinline__ uint64_t block_scan(uint64_t v, uint64_t *sh, uint64_t &total) {
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint64_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t nb = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= (uint32_t)o) inc += nb;
    }
    if (lane == 31) sh[w] = inc;
    __syncthreads();
    if (w == 0) {
        const uint64_t t = lane < nw ? sh[lane] : 0;
        uint64_t ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t nb = __shfl_up_sync(0xFFFFFFFFu, ti, o);
            if (lane >= (uint32_t)o) ti += nb;
        }
        if (lane < nw) sh[lane] = ti - t;
        if (lane == nw - 1) sh[32] = ti;
    }
    __syncthreads();
    total = sh[32];
    const uint64_t r = sh[w] + inc - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(VT) k_vmark(const VerifyParams V) {
    __shared__ uint64_t sh[33];
    for (uint64_t tile = blockIdx.x; tile < V.n_tiles; tile += gridDim.x) {
        const uint64_t i = tile * VT + threadIdx.x;
        uint32_t keep = 0;
        if (i < V.n_keys) {
            const uint64_t key = V.keys[i];
            const uint64_t p = key >> PFAC_ID_BITS;
            const uint32_t j = (uint32_t)(key & ((1u << PFAC_ID_BITS) - 1u));
            if (j < V.n_pat && p < V.n) {
                const uint32_t o0 = __ldg(V.pat_off + j), L = __ldg(V.pat_off + j + 1) - o0;
                keep = 1;
                if (L > V.trunc) {
                    // the end of p's segment: the first offset above p
                    uint32_t lo = 1, hi = V.n_seg;
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi) >> 1;
                        if (__ldg(V.seg + mid) > p) hi = mid; else lo = mid + 1;
                    }
                    const uint64_t e = __ldg(V.seg + lo);
                    if (p + L > e) {
                        keep = 0;
                    } else {
                        for (uint32_t t = V.trunc; t < L; t++)
                            if (__ldg(V.in + p + t) != __ldg(V.pat + o0 + t)) {
                                keep = 0;
                                break;
                            }
                    }
                }
            }
            V.flag[i] = (uint8_t)keep;
        }
        uint64_t total;
        block_scan(keep, sh, total);
        if (threadIdx.x == 0) V.tile_cnt[tile] = total;
    }
}

__global__ void __launch_bounds__(VT) k_vscan(const VerifyParams V) {
    __shared__ uint64_t sh[33];
    uint64_t carry = 0;
    for (uint64_t b = 0; b < V.n_tiles; b += VT) {
        const uint64_t i = b + threadIdx.x;
        const uint64_t v = i < V.n_tiles ? V.tile_cnt[i] : 0;
        uint64_t tot;
        const uint64_t ex = block_scan(v, sh, tot);
        if (i < V.n_tiles) V.tile_cnt[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *V.count = carry;
}

__global__ void __launch_bounds__(VT) k_vcompact(const VerifyParams V) {
    __shared__ uint64_t sh[33];
    for (uint64_t tile = blockIdx.x; tile < V.n_tiles; tile += gridDim.x) {
        const uint64_t i = tile * VT + threadIdx.x;
        const uint32_t keep = i < V.n_keys ? V.flag[i] : 0u;
        uint64_t total;
        const uint64_t r = block_scan(keep, sh, total);
        if (keep) V.out[V.tile_cnt[tile] + r] = V.keys[i];
    }
}

}  // namespace

extern "C" int pfac_verify(const pfac_table *t, const uint8_t *d_input, uint64_t n_bytes,
                           const uint64_t *d_seg_offsets, uint32_t n_segments,
                           const uint64_t *d_keys, uint64_t n_keys, uint64_t *d_out,
                           uint64_t *d_count, void *cuda_stream) {
    clear_error();
    if (!t || !d_count || !d_seg_offsets || (n_keys && (!d_keys || !d_out)))
        return set_error(PFAC_EINVAL, "pfac_verify: NULL argument");
    if (!t->d_blob) return set_error(PFAC_EINVAL, "pfac_verify: table was built host-only");
    const int drc = check_table_device(t, cuda_stream, "pfac_verify");
    if (drc) return drc;
    if (!t->dev.trunc || !t->dev.pat)
        return set_error(PFAC_EINVAL, "pfac_verify: the table was not built with truncate_depth");
    if (n_keys && d_keys == d_out)
        return set_error(PFAC_EINVAL, "pfac_verify: the output must not alias the candidates");
    if (n_bytes && n_segments == 0)
        return set_error(PFAC_EINVAL, "pfac_verify: a non-empty input needs a segment");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    VerifyParams V;
    memset(&V, 0, sizeof V);
    V.in = d_input;
    V.n = n_bytes;
    V.seg = d_seg_offsets;
    V.n_seg = n_segments;
    V.keys = d_keys;
    V.n_keys = n_keys;
    V.out = d_out;
    V.count = d_count;
    V.n_tiles = (n_keys + VT - 1) / VT;
    V.pat = t->dev.pat;
    V.pat_off = t->dev.pat_off;
    V.n_pat = t->dev.n_pat;
    V.trunc = t->dev.trunc;
    if (n_keys == 0) {
        const cudaError_t e = cudaMemsetAsync(d_count, 0, 8, st);
        return e == cudaSuccess ? PFAC_OK
                                : set_error(PFAC_ECUDA, "pfac_verify: %s", cudaGetErrorString(e));
    }
    void *scratch = nullptr;
    cudaError_t e = cudaMallocAsync(&scratch, V.n_tiles * 8 + n_keys + 16, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(e == cudaErrorMemoryAllocation ? PFAC_ENOMEM : PFAC_ECUDA,
                         "pfac_verify: scratch: %s", cudaGetErrorString(e));
    }
    V.tile_cnt = (uint64_t *)scratch;
    V.flag = (uint8_t *)scratch + V.n_tiles * 8;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t maxg = (uint64_t)nsm * 2;
    const uint32_t grid = (uint32_t)(V.n_tiles < maxg ? V.n_tiles : maxg);
    k_vmark<<<grid, VT, 0, st>>>(V);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_vscan<<<1, VT, 0, st>>>(V);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_vcompact<<<grid, VT, 0, st>>>(V);
        e = cudaGetLastError();
    }
    cudaFreeAsync(scratch, st);
    if (e != cudaSuccess)
        return set_error(PFAC_ECUDA, "pfac_verify: launch failed: %s", cudaGetErrorString(e));
    return PFAC_OK;
}

// Match entry points: kernel selection, workspace layout, the ordering
// kernels, and the C ABI calls pfac_workspace_bytes / pfac_match_async /
// pfac_match (Section 2.3 semantics; see include/pfac.h).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "internal.h"
#include "kernels_r.cuh"

namespace pfac {

void *scan_kernel_bps1(int, int, int, int);
void *scan_kernel_bps2(int, int, int, int);
void *scan_kernel_bps3(int, int, int, int);
void *scan_kernel_bps4(int, int, int, int);
void *scan_kernel_bps5(int, int, int, int);
void *scan_kernel_bps6(int, int, int, int);
void *scan_kernel_bps7(int, int, int, int);
void *scan_kernel_bps8(int, int, int, int);
void *scan_kernel_dense();
void *scan_kernel_r8_g0_f(int rep, int nw);
void *scan_kernel_r8_g0_fe(int rep, int nw);
void *scan_kernel_r8_g1_f(int rep, int nw);
void *scan_kernel_r8_g1_fe(int rep, int nw);
void *scan_kernel_r2_g0_f(int rep, int nw);
void *scan_kernel_r2_g0_fe(int rep, int nw);
void *scan_kernel_r2_g1_f(int rep, int nw);
void *scan_kernel_r2_g1_fe(int rep, int nw);

void *resolve_kernel(int w);
void *scan_kernel_r8_d0(int rep, int var, int nw);
void *scan_kernel_r8_d1(int rep, int var, int nw);
void *scan_kernel_r2_d0(int rep, int var, int nw);
void *scan_kernel_r2_d1(int rep, int var, int nw);

// the register-staged kernel for 8-bit or 2-bit symbols
static void *scan_kernel_r(uint32_t bps, uint32_t w, int rep, bool gram, int var, int nw) {
    if (w == 3) {  // the dense layout's transition table
        if (bps == 2) return gram ? scan_kernel_r2_d1(rep, var, nw) : scan_kernel_r2_d0(rep, var, nw);
        if (bps == 8) return gram ? scan_kernel_r8_d1(rep, var, nw) : scan_kernel_r8_d0(rep, var, nw);
        return nullptr;
    }
    if (bps == 2) {
        if (w != 0) return nullptr;  // packed records only
        if (gram) return var == VAR_FE ? scan_kernel_r2_g1_fe(rep, nw) : scan_kernel_r2_g1_f(rep, nw);
        return var == VAR_FE ? scan_kernel_r2_g0_fe(rep, nw) : scan_kernel_r2_g0_f(rep, nw);
    }
    if (bps != 8) return nullptr;
    if (gram) return var == VAR_FE ? scan_kernel_r8_g1_fe(rep, nw) : scan_kernel_r8_g1_f(rep, nw);
    return var == VAR_FE ? scan_kernel_r8_g0_fe(rep, nw) : scan_kernel_r8_g0_f(rep, nw);
}

constexpr int CHUNK = 1024;      // tiles per chunk of the key-count scan
constexpr int RT = 1024;         // threads of the scan/offset kernels

// ------------------------------------------------ segment bounds per tile --

// Validates the offsets and lists, per tile, the segment ends that the
// tile's positions can need: every o_s > tile start up to and including the
// first o_s >= tile end (at most SEG_MAXB, else SEG_OVF).
__global__ void k_bounds(const MatchParams P) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t gt = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t *seg = P.seg;
    for (uint64_t s = gt; s < P.n_seg; s += stride)
        if (__ldg(seg + s + 1) < __ldg(seg + s)) atomicOr(&P.hdr->status, ST_BADSEG);
    if (gt == 0 && (__ldg(seg) != 0 || __ldg(seg + P.n_seg) != P.n))
        atomicOr(&P.hdr->status, ST_BADSEG);
    for (uint64_t t = gt; t < P.n_tiles; t += stride) {
        const uint64_t start = t * TILE, end = start + TILE;
        uint32_t lo = 1, hi = P.n_seg;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (__ldg(seg + mid) > start) hi = mid; else lo = mid + 1;
        }
        uint32_t *B = P.tile_bounds + t * SEGW;
        uint32_t cnt = 0;
        bool ovf = false;
        for (uint32_t s = lo; s <= P.n_seg; s++) {
            const uint64_t o = __ldg(seg + s);
            if (cnt == SEG_MAXB) {
                ovf = true;
                break;
            }
            const uint64_t r = o > start ? o - start : 0;
            B[1 + cnt++] = r < 0xFFFFFFF0ull ? (uint32_t)r : 0xFFFFFFF0u;
            if (o >= end) break;
        }
        B[0] = ovf ? SEG_OVF : cnt;
    }
}

// Validates the offsets and records, per 512-byte unit of the queued scan
// kernel, the index of the first offset beyond the unit start.
__global__ void k_unitseg(const MatchParams P) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t gt = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t *seg = P.seg;
    for (uint64_t s = gt; s < P.n_seg; s += stride)
        if (__ldg(seg + s + 1) < __ldg(seg + s)) atomicOr(&P.hdr->status, ST_BADSEG);
    if (gt == 0 && (__ldg(seg) != 0 || __ldg(seg + P.n_seg) != P.n))
        atomicOr(&P.hdr->status, ST_BADSEG);
    for (uint64_t u = gt; u < P.n_tiles; u += stride) {
        const uint64_t start = u << P.unit_shift;
        uint32_t lo = 1, hi = P.n_seg;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (__ldg(seg + mid) > start) hi = mid; else lo = mid + 1;
        }
        P.unit_seg[u] = lo;
    }
}

// ------------------------------------------------ key-count scan ----------

__device__ __forceinline__ uint64_t block_excl_scan(uint64_t v, uint64_t *sh, uint64_t &total) {
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

__device__ __forceinline__ int32_t status_code(int32_t st) {
    if (st & ST_BADSEG) return PFAC_EINVAL;
    if (st & ST_TIMEOUT) return PFAC_ETIMEOUT;
    if (st & ST_DEVICE) return PFAC_EDEVICE;
    return PFAC_OK;
}

// Chunk sums of the per-tile key counts; the last CTA scans the chunk sums,
// writes the total match count and checks single-segment offsets.
__global__ void __launch_bounds__(RT) k_reduce(const MatchParams P) {
    __shared__ uint64_t sh[33];
    __shared__ bool last;
    const uint32_t c = blockIdx.x;
    uint64_t sum = 0;
    if (c < P.n_chunks) {
        const uint64_t t0 = (uint64_t)c * CHUNK;
        for (uint32_t i = threadIdx.x; i < CHUNK; i += RT) {
            const uint64_t t = t0 + i;
            if (t < P.n_tiles) sum += P.tile_k[t];
        }
    }
    uint64_t total;
    block_excl_scan(sum, sh, total);
    if (threadIdx.x == 0) {
        if (c < P.n_chunks) P.chunk[c] = total;
        __threadfence();
        last = atomicAdd(&P.hdr->done_reduce, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    uint64_t carry = 0;
    for (uint32_t base = 0; base < P.n_chunks; base += RT) {
        const uint32_t i = base + threadIdx.x;
        const uint64_t v = i < P.n_chunks ? __ldcg(P.chunk + i) : 0;
        uint64_t tot;
        const uint64_t ex = block_excl_scan(v, sh, tot);
        if (i < P.n_chunks) P.chunk[P.n_chunks + i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        *P.d_count = carry;
        if (P.n_seg <= 1) {
            const bool ok = P.n_seg == 1 ? (P.seg[0] == 0 && P.seg[1] == P.n)
                                         : (P.n == 0 && P.seg[0] == 0);
            if (!ok) atomicOr(&P.hdr->status, ST_BADSEG);
        }
    }
}

// Per-tile output offsets: chunk offset plus the scan inside the chunk.
__global__ void __launch_bounds__(RT) k_offsets(const MatchParams P) {
    __shared__ uint64_t sh[33];
    const uint32_t c = blockIdx.x;
    const uint64_t t0 = (uint64_t)c * CHUNK;
    constexpr int PER = CHUNK / RT;
    uint64_t v[PER];
    uint64_t s = 0;
#pragma unroll
    for (int i = 0; i < PER; i++) {
        const uint64_t t = t0 + threadIdx.x * PER + i;
        v[i] = t < P.n_tiles ? P.tile_k[t] : 0;
        s += v[i];
    }
    uint64_t total;
    uint64_t ex = block_excl_scan(s, sh, total) + __ldcg(P.chunk + P.n_chunks + c);
#pragma unroll
    for (int i = 0; i < PER; i++) {
        const uint64_t t = t0 + threadIdx.x * PER + i;
        if (t < P.n_tiles) P.key_off[t] = ex;
        ex += v[i];
    }
}

// Writes the keys of every tile whose records were kept; the last CTA
// publishes the call's status.
constexpr uint32_t EXPAND_THREAD_MAX = 32;  // records a single thread expands
__global__ void __launch_bounds__(256) k_expand(const MatchParams P) {
    __shared__ bool last;
    // one thread per unit: most units hold a few records or none, so the
    // units' loads are issued side by side rather than one unit per warp
    const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
    const uint32_t *pool = P.T.pool;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < P.n_tiles; t += nthr) {
        const uint32_t m = P.tile_m[t];
        if (m == 0 || m > P.unit_cap || m > EXPAND_THREAD_MAX) continue;
        uint64_t o = P.key_off[t];
        const uint64_t *rr = P.recs + t * P.unit_cap;
        const uint64_t tile_start = t << P.unit_shift;
        for (uint32_t i = 0; i < m; i++) {
            const uint64_t r = rr[i];
            const uint32_t L = fin_len_c(P, (uint32_t)r);
            const uint32_t *ids = fin_ids_c(P, (uint32_t)r);
            const uint64_t pk = (P.pos_base + tile_start + (r >> 32)) << PFAC_ID_BITS;
            for (uint32_t e = 0; e < L; e++, o++)
                if (o < P.cap) P.out[o] = pk | __ldg(ids + e);
        }
    }
    // units with more records (record space for every position): a whole
    // warp per unit, 32 records at a time, each lane's keys placed by a warp
    // scan of the records' key counts
    if (P.unit_cap > EXPAND_THREAD_MAX) {
        const uint32_t lane = threadIdx.x & 31;
        const uint64_t gwarp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const uint64_t nwarps = nthr >> 5;
        for (uint64_t t0 = gwarp * 32; t0 < P.n_tiles; t0 += nwarps * 32) {
            const uint64_t tl = t0 + lane;
            const uint32_t ml = tl < P.n_tiles ? P.tile_m[tl] : 0u;
            uint32_t dense = __ballot_sync(0xFFFFFFFFu, ml > EXPAND_THREAD_MAX && ml <= P.unit_cap);
            while (dense) {
                const uint32_t j = __ffs(dense) - 1;
                dense &= dense - 1;
                const uint64_t t = t0 + j;
                const uint32_t m = __shfl_sync(0xFFFFFFFFu, ml, j);
                uint64_t o = P.key_off[t];
                const uint64_t *rr = P.recs + t * P.unit_cap;
                const uint64_t tile_start = t << P.unit_shift;
                for (uint32_t i0 = 0; i0 < m; i0 += 32) {
                    const uint32_t i = i0 + lane;
                    uint64_t r = 0;
                    uint32_t L = 0;
                    if (i < m) {
                        r = rr[i];
                        L = fin_len_c(P, (uint32_t)r);
                    }
                    uint32_t inc = L;
#pragma unroll
                    for (int s = 1; s < 32; s <<= 1) {
                        const uint32_t nb = __shfl_up_sync(0xFFFFFFFFu, inc, s);
                        if (lane >= (uint32_t)s) inc += nb;
                    }
                    if (L) {
                        const uint32_t *ids = fin_ids_c(P, (uint32_t)r);
                        const uint64_t pk = (P.pos_base + tile_start + (r >> 32)) << PFAC_ID_BITS;
                        uint64_t oo = o + inc - L;
                        for (uint32_t e = 0; e < L; e++, oo++)
                            if (oo < P.cap) P.out[oo] = pk | __ldg(ids + e);
                    }
                    o += __shfl_sync(0xFFFFFFFFu, inc, 31);
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&P.hdr->done_expand, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0 && P.d_status) {
        __threadfence();
        *P.d_status = status_code(*(volatile int32_t *)&P.hdr->status);
    }
}

// ------------------------------------------------ host side ---------------

struct Plan {
    int var;
    uint32_t k;
    uint32_t tbl_words, tbl_c_words, tbl_e_words, tbl_m_words;
    uint32_t rep_log2;
    uint32_t tbl_g_words, g_rep, g_fold;  // gram filter: words (all copies), copies, fold
    uint32_t tbl_b_words;                 // prefix bytes as the first stage
    uint32_t nw;                          // warps per CTA of the queued kernel
    uint32_t dense_rows;
    uint32_t unit_shift, unit_cap;
    void *kernel;       // scan pass
    void *kernel_emit;  // emit pass
    size_t smem;
    bool queued;
    int kind;           // SCAN_QUEUED or SCAN_REGISTER (compressed layout)
    bool defer;         // the scan hands whole-slice queues to the resolver kernel
    void *kernel_res;
    // emit pass of a register-staged plan: the queued kernel with tables of
    // its own (one bitmap copy, entries through L2)
    size_t smem_emit;
    uint32_t e_tbl_words, e_tbl_m_words;
};

enum { SCAN_QUEUED = 1, SCAN_REGISTER = 2, SCAN_SERIAL = 3 };

struct WsLayout {
    uint64_t hdr, tile_m, tile_k, key_off, chunk, ovf, recs, bounds, defer, dbatch, total;
    uint32_t n_tiles, n_chunks, defer_cap, dbatch_cap;
};

// entries per slice the resolver kernel's buffer holds (more go to the
// scan kernel's own resolution)
constexpr uint32_t DEFER_PER_UNIT = 8;

static inline uint64_t al256(uint64_t x) { return (x + 255) & ~255ull; }

static WsLayout ws_layout(uint64_t n_bytes, uint32_t n_seg, const Plan &pl) {
    WsLayout L{};
    const uint64_t ub = 1ull << pl.unit_shift;
    const uint64_t nt = (n_bytes + ub - 1) / ub;
    L.n_tiles = (uint32_t)nt;
    L.n_chunks = (uint32_t)((nt + CHUNK - 1) / CHUNK);
    uint64_t o = 0;
    auto put = [&](uint64_t sz) {
        const uint64_t at = o;
        o = al256(o + sz);
        return at;
    };
    L.hdr = put(sizeof(WsHeader));
    L.tile_m = put(nt * 4);
    L.tile_k = put(nt * 8);
    L.key_off = put(nt * 8);
    L.chunk = put((uint64_t)L.n_chunks * 16);
    L.ovf = put(nt * 4);
    L.recs = put(nt * pl.unit_cap * 8);
    // segment data: per-tile lists (tile-synchronous kernel) or the first
    // offset index per unit (queued kernel)
    L.bounds = put(n_seg > 1 ? (pl.queued ? nt * 4 : nt * SEGW * 4) : 0);
    // register-staged plans: the queues handed to the resolver kernel (at
    // most one batch per slice, plus each warp's last)
    const uint64_t dcap = pl.defer ? std::min<uint64_t>(nt * DEFER_PER_UNIT, 0xFFFFFF00ull) : 0;
    L.defer_cap = (uint32_t)dcap;
    L.dbatch_cap = pl.defer ? (uint32_t)std::min<uint64_t>(nt + 4096, 0xFFFFFF00ull) : 0u;
    L.defer = put(dcap * 16);
    L.dbatch = put((uint64_t)L.dbatch_cap * 8);
    L.total = o;
    return L;
}

static void *scan_kernel_for(uint32_t bps, int var, int emit, int nw, int w) {
    switch (bps) {
        case 1: return scan_kernel_bps1(var, emit, nw, w);
        case 2: return scan_kernel_bps2(var, emit, nw, w);
        case 3: return scan_kernel_bps3(var, emit, nw, w);
        case 4: return scan_kernel_bps4(var, emit, nw, w);
        case 5: return scan_kernel_bps5(var, emit, nw, w);
        case 6: return scan_kernel_bps6(var, emit, nw, w);
        case 7: return scan_kernel_bps7(var, emit, nw, w);
        case 8: return scan_kernel_bps8(var, emit, nw, w);
        default: return nullptr;
    }
}

static size_t dense_smem(uint32_t tbl_words) {
    const size_t tbl = ((size_t)tbl_words * 4 + 127) & ~(size_t)127;
    return tbl + STAGES * STAGE_IN + STAGES * SEGW * 4 + 2 * STAGES * 8 + 2 * STAGES * 4 +
           (CW + 1) * 8;
}

constexpr size_t SMEM_LIMIT = 232448;  // per-CTA dynamic shared memory on sm_103a

static size_t queued_smem(uint64_t words, uint32_t nw = QW) {
    const size_t tbl = ((size_t)words * 4 + 127) & ~(size_t)127;
    return tbl + nw * sizeof(WarpArea);
}

// Shared-memory wavefronts of one warp-wide bitmap load with 2^rep copies
// (interleaved word by word): lanes sharing a copy collide on a bank.
static double load_wavefronts(int rep) {
    static const double wf[6] = {3.7, 3.4, 3.1, 2.85, 2.0, 1.0};
    return wf[rep < 0 ? 0 : (rep > 5 ? 5 : rep)];
}

// Estimated warp instructions per 512-byte slice of a first stage that
// passes a share `dens` of the positions (measured orders of magnitude:
// ~9 per tested position row, 2 more for hashing, bank-conflict replays,
// ~90 for a slice with any candidate and ~12 per candidate).
static double first_stage_cost(double dens, int rep, bool hashed) {
    const double cand = dens * 512.0;
    return (hashed ? 176.0 : 144.0) + 48.0 * (load_wavefronts(rep) - 1.0) +
           90.0 * (1.0 - exp(-cand)) + 12.0 * cand;
}

// Estimated SM cycles per slice of the register-staged kernel beyond a fixed
// part: the first stage's shared-memory wavefronts (16 lookups a lane) and
// about 10 cycles per candidate for the second stage (a fit to the alphabet-
// 256 cell with 1,000 patterns: 112 cycles a slice with the gram filter at
// 0.1% candidates and 3.7 wavefronts a lookup, 157 with the prefix bitmap in
// 16 copies at 1.5% and 2 wavefronts), plus a little for the gram hash.
static double r_cost(double dens, int rep, bool hashed) {
    return 16.0 * load_wavefronts(rep) + 10.0 * 512.0 * dens + (hashed ? 4.0 : 0.0);
}

static size_t r_smem(uint64_t words, uint32_t nw = RNW) {
    return (((size_t)words * 4 + 127) & ~(size_t)127) + nw * sizeof(RWarpArea);
}

constexpr int R_MAX_REP = 4;  // copies of the first-stage bitmap: 1 .. 16
constexpr bool R_BY_DEFAULT = true;  // the register-staged kernel by default for 8-bit symbols

// Plan of the register-staged kernel (8-bit symbols): the first stage (the
// prefix bitmap, or the gram filter folded to fit) and its copies, entries
// and child masks in shared memory as they fit, chosen by r_cost; the emit
// pass runs the queued kernel with one bitmap copy.
static int make_plan_r(const pfac_table *t, uint32_t k, int var, uint32_t masks, uint32_t gram,
                       int want, uint32_t nw, Plan *pl) {
    const DevTable &T = t->dev;
    const uint64_t ent = 1ull << (k * T.bps);
    const uint32_t fw = (uint32_t)(ent >= 32 ? ent / 32 : 1);
    const uint32_t cw = (fw + (1u << T.c_shift[k]) - 1) >> T.c_shift[k];
    const uint32_t ew = T.n_e[k];
    const bool have_m = T.M[k] != nullptr;
    const uint32_t mw = T.m_words[k];
    const double dens_f = (double)ew / (double)ent;
    double best = 1e30;
    int b_var = 0, b_rep = -1;
    uint32_t b_fold = 0;
    bool b_gram = false, b_m = false;
    for (int vv = VAR_FE; vv >= VAR_F; vv--) {
        if (var != 0 && var != vv) continue;
        for (int mm = 1; mm >= 0; mm--) {
            const bool mon = mm == 1;
            if (mon && !(have_m && masks != 1)) continue;
            if (!mon && masks == 2) continue;
            const uint64_t base = cw + (vv == VAR_FE ? ew : 0u) + (mon ? mw : 0u);
            // a preference for what keeps the walks short: entries in shared
            // memory, and above all the child masks, which drop most candidates
            const double bias = (vv == VAR_FE ? 1.0 : 1.05) * (mon ? 1.0 : 1.3);
            for (int r = 0; r <= R_MAX_REP; r++) {
                if (want >= 0 && r != want) continue;
                if (gram != 2 && r_smem(base + ((uint64_t)fw << r), nw) <= SMEM_LIMIT) {
                    const double c = r_cost(dens_f, r, false) * bias;
                    if (c < best) {
                        best = c;
                        b_var = vv;
                        b_rep = r;
                        b_gram = false;
                        b_m = mon;
                    }
                }
                if (T.g_len && gram != 1) {
                    const uint32_t hb = T.g_bits;
                    const uint64_t gw0 = (1ull << hb) / 32;
                    for (uint32_t f = 0; hb - f >= GRAM_MIN_BITS; f++) {
                        if (r_smem(base + fw + ((gw0 >> f) << r), nw) > SMEM_LIMIT) continue;
                        const double dens = 1.0 - exp(-(double)T.g_set / (double)(1ull << (hb - f)));
                        const double c = r_cost(dens, r, true) * bias;
                        if ((gram == 2 || dens < 0.5) && c < best) {
                            best = c;
                            b_var = vv;
                            b_rep = r;
                            b_gram = true;
                            b_fold = f;
                            b_m = mon;
                        }
                        break;  // the least folding that fits
                    }
                }
            }
        }
    }
    if (b_rep < 0)
        return set_error(PFAC_EINVAL, "pfac_match: no register-staged plan fits in shared memory "
                         "with depth %u%s", k, want >= 0 ? " and these copies" : "");
    pl->var = b_var;
    pl->k = k;
    pl->tbl_c_words = cw;
    pl->tbl_e_words = b_var == VAR_FE ? ew : 0u;
    pl->tbl_m_words = b_m ? mw : 0u;
    pl->tbl_b_words = 0;
    if (b_gram) {
        pl->rep_log2 = 0;
        pl->tbl_words = fw;
        pl->g_rep = (uint32_t)b_rep;
        pl->g_fold = b_fold;
        pl->tbl_g_words = (uint32_t)((((1ull << T.g_bits) / 32) >> b_fold) << b_rep);
    } else {
        pl->rep_log2 = (uint32_t)b_rep;
        pl->tbl_words = fw << b_rep;
    }
    pl->nw = nw;
    pl->kind = SCAN_REGISTER;
    pl->kernel = scan_kernel_r(T.bps, T.W, b_rep, b_gram, b_var, (int)nw);
    pl->defer = true;
    pl->kernel_res = resolve_kernel((int)T.W);
    pl->smem = r_smem((uint64_t)pl->tbl_words + pl->tbl_c_words + pl->tbl_e_words +
                      pl->tbl_m_words + pl->tbl_g_words, nw);
    // the emit pass: the queued kernel, one bitmap copy, entries through L2,
    // child masks when they fit beside its warps' rings
    pl->e_tbl_words = fw;
    pl->e_tbl_m_words = (have_m && queued_smem((uint64_t)fw + cw + mw, QW) <= SMEM_LIMIT) ? mw : 0u;
    pl->smem_emit = queued_smem((uint64_t)fw + cw + pl->e_tbl_m_words, QW);
    pl->kernel_emit = scan_kernel_for(T.bps, VAR_F, 1, QW, (int)T.W);
    pl->unit_shift = SLICE_SHIFT;
    pl->unit_cap = SCAP;
    pl->queued = true;
    if (!pl->kernel || !pl->kernel_emit || !pl->kernel_res)
        return set_error(PFAC_EINVAL, "pfac_match: no register-staged kernel for this table");
    return PFAC_OK;
}

static int make_plan(const pfac_table *t, const pfac_match_opts *opts, Plan *pl) {
    const DevTable &T = t->dev;
    memset(pl, 0, sizeof(*pl));
    // the dense layout runs the compressed layout's kernels over its
    // transition table (record format 3), or on request the thread-serial
    // kernel (scan_kernel 3)
    if (T.layout == PFAC_LAYOUT_DENSE && opts && opts->scan_kernel == SCAN_SERIAL) {
        pl->kind = SCAN_SERIAL;
        pl->var = VAR_DENSE;
        uint32_t rows = (uint32_t)(TABLE_SMEM_MAX / (4ull * T.sigma));
        if (rows > T.n_nodes) rows = T.n_nodes;
        pl->dense_rows = rows;
        pl->tbl_words = rows * T.sigma;
        pl->kernel = pl->kernel_emit = scan_kernel_dense();
        pl->smem = dense_smem(pl->tbl_words);
        pl->unit_shift = 13;
        pl->unit_cap = REC_CAP;
        pl->queued = false;
        return PFAC_OK;
    }
    const uint32_t k = opts && opts->prefix_depth ? opts->prefix_depth
                                                   : (t->tuned_k ? t->tuned_k : T.kdef);
    if (k < t->kmin || k > t->kmax)
        return set_error(PFAC_EINVAL, "pfac_match: prefix depth %u not held (table holds %u..%u)",
                         k, t->kmin, t->kmax);
    const uint64_t ent = 1ull << (k * T.bps);
    const uint32_t fw = (uint32_t)(ent >= 32 ? ent / 32 : 1);
    const uint32_t cw = (fw + (1u << T.c_shift[k]) - 1) >> T.c_shift[k];
    const uint32_t ew = T.n_e[k];
    int var = opts && opts->variant ? (int)opts->variant
                                    : (t->tuned_variant ? (int)t->tuned_variant : 0);
    // the table's tuned choice applies only when the caller picks neither the
    // variant nor the depth
    const bool use_tuned = !(opts && (opts->variant || opts->prefix_depth));
    const uint32_t nwant = opts && opts->warps_per_cta ? opts->warps_per_cta
                                                      : (use_tuned && t->tuned_nw ? t->tuned_nw : QW);
    if (nwant != QW && nwant != QW_WIDE)
        return set_error(PFAC_EINVAL, "pfac_match: warps_per_cta %u (16 or 24)", nwant);
    const uint32_t masks = opts && opts->child_masks ? opts->child_masks
                                                    : (use_tuned ? t->tuned_masks : 0u);
    if (masks > 2) return set_error(PFAC_EINVAL, "pfac_match: child_masks %u", masks);
    const bool have_m = T.M[k] != nullptr;
    const uint32_t mw = T.m_words[k];  // words of the packed child masks
    if (masks == 2 && !have_m)
        return set_error(PFAC_EINVAL, "pfac_match: depth %u keeps no child masks (too many "
                         "entries for shared memory)", k);
    const uint32_t gram = opts && opts->gram_filter ? opts->gram_filter
                                                   : (use_tuned ? t->tuned_gram : 0u);
    if (gram > 2) return set_error(PFAC_EINVAL, "pfac_match: gram_filter %u", gram);
    if (gram == 2 && !T.g_len)
        return set_error(PFAC_EINVAL, "pfac_match: the table has no gram filter");
    const uint32_t pbytes = opts && opts->prefix_bytes ? opts->prefix_bytes
                                                      : (use_tuned ? t->tuned_bytes : 0u);
    if (pbytes > 2) return set_error(PFAC_EINVAL, "pfac_match: prefix_bytes %u", pbytes);
    if (pbytes == 2 && !T.B[k])
        return set_error(PFAC_EINVAL, "pfac_match: depth %u has no prefix bytes (more than %u "
                         "index bits)", k, BYTES_MAX_BITS);
    if (pbytes == 2 && gram == 2)
        return set_error(PFAC_EINVAL, "pfac_match: prefix bytes and the gram filter exclude "
                         "each other");
    const uint32_t copies = opts && opts->bitmap_copies ? opts->bitmap_copies
                                                       : (use_tuned ? t->tuned_copies : 0u);
    int want = -1;
    if (copies) {
        want = 0;
        while ((1u << want) < copies) want++;
        if ((1u << want) != copies || want > 5)
            return set_error(PFAC_EINVAL, "pfac_match: bitmap_copies %u is not 1, 2, 4, .., 32",
                             copies);
    }
    if (pbytes == 2 && copies > 1)
        return set_error(PFAC_EINVAL, "pfac_match: prefix bytes take one bitmap copy (%u asked)",
                         copies);
    if (var != 0 && var != VAR_F && var != VAR_FE)
        return set_error(PFAC_EINVAL, "pfac_match: unknown variant %d", var);
    // a merged trie (reduction step 2) runs the queued kernel's merged-trie
    // instance: entries through L2, the default CTA width
    if (T.dag && var == VAR_FE)
        return set_error(PFAC_EINVAL, "pfac_match: a merged trie takes variant 1 (entries in L2)");
    if (T.dag && nwant != QW)
        return set_error(PFAC_EINVAL, "pfac_match: a merged trie takes %u warps per CTA", QW);
    if (T.dag) var = VAR_F;

    // ---- records kept per slice: 32, or 512 (one per position, so that no
    // slice is scanned twice) where many matches are likely
    const uint32_t recs = opts && opts->records_per_slice
                              ? opts->records_per_slice
                              : (use_tuned && t->tuned_records
                                     ? t->tuned_records
                                     : (t->match_density * SLICE > 8.0 ? (uint32_t)SLICE : SCAP));
    if (recs != (uint32_t)SCAP && recs != (uint32_t)SLICE)
        return set_error(PFAC_EINVAL, "pfac_match: records_per_slice %u (32 or 512)", recs);
    const uint32_t resolver = opts && opts->resolver
                                  ? opts->resolver
                                  : (use_tuned ? t->tuned_resolver : 0u);
    if (resolver > 2) return set_error(PFAC_EINVAL, "pfac_match: resolver %u", resolver);
    if (resolver == 2 && T.dag)
        return set_error(PFAC_EINVAL, "pfac_match: a merged trie resolves its queues in the scan");
    // by default the resolver kernel takes the queues where at least four
    // windows per slice pass the prefix bitmap (uniform text): with fewer,
    // its launch costs more than the scan saves
    const bool defer = !T.dag && (resolver == 2 ||
                                  (resolver == 0 && (double)ew * SLICE >= 4.0 * (double)ent));

    // ---- the register-staged kernel (8-bit symbols): on request, or by
    // default when the caller asks for nothing only the queued kernel has
    const uint32_t want_kind = opts && opts->scan_kernel ? opts->scan_kernel
                                                         : (use_tuned ? t->tuned_kernel : 0u);
    if (want_kind > 2)
        return set_error(PFAC_EINVAL, "pfac_match: scan_kernel %u (3: dense layout only)", want_kind);
    const bool r_usable = (T.bps == 8 || T.bps == 2) && pbytes != 2 && !T.dag;
    if (want_kind == SCAN_REGISTER && !r_usable)
        return set_error(PFAC_EINVAL, "pfac_match: the register-staged kernel needs 8-bit or 2-bit "
                         "symbols (alphabets of 129 to 256, or of up to 4), no prefix bytes and "
                         "no merged trie");
    if (want_kind == SCAN_REGISTER || (want_kind == 0 && r_usable && T.bps == 8 && R_BY_DEFAULT)) {
        const uint32_t rnw = opts && opts->warps_per_cta
                                 ? opts->warps_per_cta
                                 : (use_tuned && t->tuned_nw ? t->tuned_nw : (uint32_t)RNW);
        const int rc = make_plan_r(t, k, var, masks, gram, want, rnw, pl);
        pl->unit_cap = recs;
        pl->defer = defer;
        if (rc == PFAC_OK || want_kind == SCAN_REGISTER) return rc;
        clear_error();
        memset(pl, 0, sizeof(*pl));
    }

    // ---- prefix bitmap as the first stage: largest replication that fits
    auto best_rep = [&](uint64_t extra) -> int {
        int rep = -1;
        for (int r = 0; r <= 5; r++)
            if (queued_smem(((uint64_t)fw << r) + cw + extra, nwant) <= SMEM_LIMIT) rep = r;
        return rep;
    };
    int var_f = var;
    if (var_f == 0) {
        const int rep_f = best_rep(0), rep_fe = best_rep(ew);
        var_f = (rep_fe >= 0 && rep_fe >= rep_f - 1) ? VAR_FE : VAR_F;
    }
    const uint32_t e_f = var_f == VAR_FE ? ew : 0u;
    // child masks: with them if they fit (or on request), then the most copies
    const bool m_f = have_m && (masks == 2 || (masks == 0 && best_rep(e_f + mw) >= 0));
    int rep_f = best_rep(e_f + (m_f ? mw : 0u));
    if (want >= 0 && want <= rep_f) rep_f = want;
    else if (want >= 0) rep_f = -2;  // the requested copies do not fit
    const double dens_f = (double)ew / (double)ent;

    // ---- gram filter as the first stage: the prefix bitmap once (for the
    // exact test of survivors), the filter folded (adjacent words OR-ed)
    // until the chosen copies fit
    bool use_g = false;
    int var_g = 0, rep_g = -1;
    uint32_t fold_g = 0;
    bool m_g = false;
    double cost_g = 1e30;
    if (T.g_len && gram != 1) {
        const uint32_t hb = T.g_bits;
        const uint64_t gw0 = (1ull << hb) / 32;
        // entries and child masks in shared memory compete with the filter's
        // bits: every allowed combination is costed, keeping them when that
        // costs little
        for (int vv = VAR_FE; vv >= VAR_F; vv--) {
            if (var != 0 && var != vv) continue;
            for (int mm = 1; mm >= 0; mm--) {
                const bool mon = mm == 1;
                if (mon && !(have_m && masks != 1)) continue;
                if (!mon && masks == 2) continue;
                const uint64_t base = fw + cw + (vv == VAR_FE ? ew : 0u) + (mon ? mw : 0u);
                // a small preference for what keeps the walks short
                const double bias = (vv == VAR_FE ? 1.0 : 1.05) * (mon ? 1.0 : 1.1);
                for (int r = 0; r <= 5; r++) {
                    if (want >= 0 && r != want) continue;
                    for (uint32_t f = 0; hb - f >= GRAM_MIN_BITS; f++) {
                        if (queued_smem(base + ((gw0 >> f) << r), nwant) > SMEM_LIMIT) continue;
                        // expected share of positions through the first stage
                        const double dens =
                            1.0 - exp(-(double)T.g_set / (double)(1ull << (hb - f)));
                        const double c = first_stage_cost(dens, r, true) * bias;
                        if ((gram == 2 || dens < 0.5) && c < cost_g) {
                            cost_g = c;
                            rep_g = r;
                            fold_g = f;
                            var_g = vv;
                            m_g = mon;
                        }
                        break;  // the least folding that fits
                    }
                }
            }
        }
        if (rep_g >= 0) {
            const double cost_f =
                rep_f >= 0 ? first_stage_cost(dens_f, rep_f, false) * (m_f ? 1.0 : 1.1) : 1e30;
            use_g = gram == 2 || cost_g < cost_f;
        } else if (gram == 2) {
            return set_error(PFAC_EINVAL, "pfac_match: the gram filter does not fit in shared "
                             "memory with depth %u%s", k, want >= 0 ? " and these copies" : "");
        }
    }
    // ---- prefix bytes as the first stage (one copy): the prefix bitmap once
    // for ranks, then entries and child masks as they fit.  By default for
    // prefix nodes whose bitmap passes at least 1% of the positions (where
    // the cheaper second stage pays), unless the gram filter is chosen.
    bool use_b = false;
    int var_b = 0;
    bool m_b = false;
    if (T.B[k] && pbytes != 1 && gram != 2 && (want <= 0)) {
        const uint64_t bw = ent / 4;
        for (int vv = VAR_FE; vv >= VAR_F && !use_b; vv--) {
            if (var != 0 && var != vv) continue;
            for (int mm = 1; mm >= 0; mm--) {
                const bool mon = mm == 1;
                if (mon && !(have_m && masks != 1)) continue;
                if (!mon && masks == 2) continue;
                if (queued_smem(bw + fw + cw + (vv == VAR_FE ? ew : 0u) + (mon ? mw : 0u),
                                nwant) <= SMEM_LIMIT) {
                    var_b = vv;
                    m_b = mon;
                    use_b = pbytes == 2 || (!use_g && dens_f >= 0.01);
                    break;
                }
            }
        }
        if (pbytes == 2 && !use_b)
            return set_error(PFAC_EINVAL, "pfac_match: prefix bytes of depth %u do not fit in "
                             "shared memory", k);
    }
    if (use_b) {
        use_g = false;
        var = var_b;
        pl->rep_log2 = 0;
        pl->tbl_words = fw;
        pl->tbl_e_words = var == VAR_FE ? ew : 0u;
        pl->tbl_m_words = m_b ? mw : 0u;
        pl->tbl_b_words = (uint32_t)(ent / 4);
    } else if (use_g) {
        var = var_g;
        pl->rep_log2 = 0;
        pl->tbl_words = fw;
        pl->tbl_e_words = var == VAR_FE ? ew : 0u;
        pl->tbl_m_words = m_g ? mw : 0u;
        pl->g_rep = (uint32_t)rep_g;
        pl->g_fold = fold_g;
        pl->tbl_g_words = (uint32_t)((((1ull << T.g_bits) / 32) >> fold_g) << rep_g);
    } else {
        if (rep_f == -2)
            return set_error(PFAC_EINVAL, "pfac_match: %u bitmap copies do not fit", copies);
        if (rep_f < 0)
            return set_error(PFAC_EINVAL, "pfac_match: prefix node of depth %u does not fit in "
                             "shared memory with variant %d%s", k, var_f,
                             m_f ? " and child masks" : "");
        var = var_f;
        pl->rep_log2 = (uint32_t)rep_f;
        pl->tbl_words = (uint32_t)((uint64_t)fw << rep_f);
        pl->tbl_e_words = e_f;
        pl->tbl_m_words = m_f ? mw : 0u;
    }
    pl->var = var;
    pl->k = k;
    pl->tbl_c_words = cw;
    // a wider CTA on request, when the tables leave room for its warps
    const uint64_t tw = (uint64_t)pl->tbl_b_words + pl->tbl_words + pl->tbl_c_words +
                        pl->tbl_e_words + pl->tbl_m_words + pl->tbl_g_words;
    if (queued_smem(tw, nwant) > SMEM_LIMIT)
        return set_error(PFAC_EINVAL, "pfac_match: %u warps do not fit next to the tables", nwant);
    pl->nw = nwant;
    pl->kind = SCAN_QUEUED;
    // the resolver kernel takes the plain tries' queues (the merged trie's
    // walk stays in its own instance)
    pl->defer = defer;
    pl->kernel_res = pl->defer ? resolve_kernel((int)T.W) : nullptr;
    const int kvar = T.dag ? (VAR_F | VAR_MERGED) : var;
    pl->kernel = scan_kernel_for(T.bps, kvar, 0, (int)nwant, (int)T.W);
    pl->kernel_emit = scan_kernel_for(T.bps, kvar, 1, (int)nwant, (int)T.W);
    pl->smem = queued_smem(tw, nwant);
    pl->unit_shift = SLICE_SHIFT;
    pl->unit_cap = recs;
    pl->queued = true;
    if (!pl->kernel || !pl->kernel_emit || (pl->defer && !pl->kernel_res))
        return set_error(PFAC_EINVAL, "pfac_match: no kernel for this table");
    return PFAC_OK;
}

static std::mutex g_attr_mu;

static int prepare_kernel(void *fn, size_t smem) {
    // raise the dynamic shared-memory limit once per kernel, device and size
    static void *done_fn[128];
    static int done_dev[128];
    static size_t done_sz[128];
    static int n_done = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_attr_mu);
    for (int i = 0; i < n_done; i++)
        if (done_fn[i] == fn && done_dev[i] == dev && done_sz[i] >= smem) return PFAC_OK;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return set_error(PFAC_ECUDA, "pfac_match: smem attribute: %s", cudaGetErrorString(e));
    if (n_done < 128) {
        done_fn[n_done] = fn;
        done_dev[n_done] = dev;
        done_sz[n_done] = smem;
        n_done++;
    }
    return PFAC_OK;
}

int check_table_device(const pfac_table *t, void *cuda_stream, const char *who) {
    int cur = 0;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess)
        return set_error(PFAC_ECUDA, "%s: cudaGetDevice: %s", who, cudaGetErrorString(e));
    if (cur != t->device)
        return set_error(PFAC_EINVAL, "%s: the current device is %d but the table lives on "
                         "device %d; make device %d current", who, cur, t->device, t->device);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cuda_stream && cudaStreamIsCapturing((cudaStream_t)cuda_stream, &cap) != cudaSuccess) {
        cudaGetLastError();
        cap = cudaStreamCaptureStatusNone;
    }
    // the stream's device cannot be queried while the stream captures a graph
    // (the query is not permitted then); the current-device check stands
    if (cuda_stream && cap == cudaStreamCaptureStatusNone) {
        int sd = 0;
        e = cudaStreamGetDevice((cudaStream_t)cuda_stream, &sd);
        if (e != cudaSuccess)
            return set_error(PFAC_ECUDA, "%s: cudaStreamGetDevice: %s", who,
                             cudaGetErrorString(e));
        if (sd != t->device)
            return set_error(PFAC_EINVAL, "%s: the stream belongs to device %d but the table "
                             "lives on device %d", who, sd, t->device);
    }
    return PFAC_OK;
}

static int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

}  // namespace pfac

using namespace pfac;

extern "C" int pfac_workspace_bytes(const pfac_table *t, uint64_t n_bytes, uint32_t n_segments,
                                    const pfac_match_opts *opts, uint64_t *bytes) {
    if (!t || !bytes) return set_error(PFAC_EINVAL, "pfac_workspace_bytes: NULL argument");
    if (n_bytes >> (64 - PFAC_ID_BITS))
        return set_error(PFAC_EINVAL, "pfac_workspace_bytes: input longer than 2^%d bytes",
                         64 - PFAC_ID_BITS);
    Plan pl;
    const int rc = make_plan(t, opts, &pl);
    if (rc) return rc;
    *bytes = ws_layout(n_bytes, n_segments, pl).total;
    return PFAC_OK;
}

extern "C" int pfac_match_plan(const pfac_table *t, const pfac_match_opts *opts,
                               pfac_plan_info *out) {
    clear_error();
    if (!t || !out) return set_error(PFAC_EINVAL, "pfac_match_plan: NULL argument");
    Plan pl;
    const int rc = make_plan(t, opts, &pl);
    if (rc) return rc;
    memset(out, 0, sizeof *out);
    out->smem_bytes = (uint32_t)pl.smem;
    if (!pl.queued) return PFAC_OK;
    out->variant = (uint32_t)pl.var;
    out->prefix_depth = pl.k;
    const bool g = pl.tbl_g_words != 0;
    out->bitmap_copies = 1u << (g ? pl.g_rep : pl.rep_log2);
    out->child_masks = pl.tbl_m_words ? 2u : 1u;
    out->gram_filter = g ? 2u : 1u;
    out->gram_bits = g ? t->dev.g_bits - pl.g_fold : 0u;
    out->prefix_bytes = pl.tbl_b_words ? 2u : 1u;
    out->warps_per_cta = pl.nw;
    out->scan_kernel = (uint32_t)pl.kind;
    out->records_per_slice = pl.unit_cap;
    out->resolver = pl.kind == SCAN_SERIAL ? 0u : (pl.defer ? 2u : 1u);
    return PFAC_OK;
}

extern "C" int pfac_match_async(const pfac_table *t, const uint8_t *d_input, uint64_t n_bytes,
                                const uint64_t *d_seg_offsets, uint32_t n_segments,
                                uint64_t *d_out_keys, uint64_t out_capacity, uint64_t *d_count,
                                int32_t *d_status, void *d_workspace, uint64_t workspace_bytes,
                                const pfac_match_opts *opts, void *cuda_stream) {
    if (!t || !d_count || !d_seg_offsets || !d_workspace)
        return set_error(PFAC_EINVAL, "pfac_match: NULL argument");
    if (!t->d_blob) return set_error(PFAC_EINVAL, "pfac_match: table was built host-only");
    {
        const int drc = check_table_device(t, cuda_stream, "pfac_match");
        if (drc) return drc;
    }
    if (n_bytes && !d_input) return set_error(PFAC_EINVAL, "pfac_match: NULL input");
    if (((uintptr_t)d_input & 15) != 0)
        return set_error(PFAC_EINVAL, "pfac_match: input must be 16-byte aligned");
    if (((uintptr_t)d_workspace & 255) != 0)
        return set_error(PFAC_EINVAL, "pfac_match: workspace must be 256-byte aligned");
    if (n_bytes >> (64 - PFAC_ID_BITS))
        return set_error(PFAC_EINVAL, "pfac_match: input longer than 2^%d bytes", 64 - PFAC_ID_BITS);
    if (n_bytes && n_segments == 0)
        return set_error(PFAC_EINVAL, "pfac_match: a non-empty input needs a segment");
    if (out_capacity && !d_out_keys) return set_error(PFAC_EINVAL, "pfac_match: NULL output");
    const uint64_t starts_end = opts && opts->starts_end ? opts->starts_end : n_bytes;
    const uint64_t pos_base = opts ? opts->position_base : 0;
    if (starts_end > n_bytes)
        return set_error(PFAC_EINVAL, "pfac_match: starts_end %llu beyond the input",
                         (unsigned long long)starts_end);
    if ((pos_base + n_bytes) >> (64 - PFAC_ID_BITS) || pos_base + n_bytes < pos_base)
        return set_error(PFAC_EINVAL, "pfac_match: position_base + n_bytes reaches 2^%d",
                         64 - PFAC_ID_BITS);
    Plan pl;
    int rc = make_plan(t, opts, &pl);
    if (rc) return rc;
    const WsLayout L = ws_layout(n_bytes, n_segments, pl);
    if (workspace_bytes < L.total)
        return set_error(PFAC_EINVAL, "pfac_match: workspace of %llu bytes, %llu needed",
                         (unsigned long long)workspace_bytes, (unsigned long long)L.total);
    const bool reg = pl.kind == SCAN_REGISTER;
    const size_t smem_emit = reg ? pl.smem_emit : pl.smem;
    rc = prepare_kernel(pl.kernel, pl.smem);
    if (!rc && pl.kernel_emit != pl.kernel) rc = prepare_kernel(pl.kernel_emit, smem_emit);
    if (rc) return rc;

    cudaStream_t st = (cudaStream_t)cuda_stream;
    uint8_t *W = (uint8_t *)d_workspace;
    MatchParams P;
    memset(&P, 0, sizeof(P));
    P.T = t->dev;
    P.in = d_input;
    P.n = n_bytes;
    P.seg = d_seg_offsets;
    P.n_seg = n_segments;
    // units holding a start position (the rest of the input is halo)
    const uint64_t ub = 1ull << pl.unit_shift;
    P.n_tiles = (uint32_t)((starts_end + ub - 1) >> pl.unit_shift);
    P.starts_end = starts_end;
    P.pos_base = pos_base;
    P.out = d_out_keys;
    P.cap = out_capacity;
    P.d_count = d_count;
    P.d_status = d_status;
    P.hdr = (WsHeader *)(W + L.hdr);
    P.tile_m = (uint32_t *)(W + L.tile_m);
    P.tile_k = (uint64_t *)(W + L.tile_k);
    P.key_off = (uint64_t *)(W + L.key_off);
    P.chunk = (uint64_t *)(W + L.chunk);
    P.n_chunks = (uint32_t)((P.n_tiles + CHUNK - 1) / CHUNK);
    P.ovf_list = (uint32_t *)(W + L.ovf);
    P.recs = (uint64_t *)(W + L.recs);
    P.tile_bounds = (uint32_t *)(W + L.bounds);
    P.unit_seg = (uint32_t *)(W + L.bounds);
    P.unit_shift = pl.unit_shift;
    P.unit_cap = pl.unit_cap;
    P.k = pl.k;
    P.F = pl.k ? t->dev.F[pl.k] : nullptr;
    P.C = pl.k ? t->dev.C[pl.k] : nullptr;
    P.E = pl.k ? t->dev.E[pl.k] : nullptr;
    P.M = pl.k ? t->dev.M[pl.k] : nullptr;
    P.c_shift = pl.k ? t->dev.c_shift[pl.k] : 0u;
    P.tbl_m_words = pl.tbl_m_words;
    P.tbl_g_words = pl.tbl_g_words;
    P.g_rep = pl.g_rep;
    P.g_fold = pl.g_fold;
    P.g_hb = pl.tbl_g_words ? t->dev.g_bits - pl.g_fold : 0u;
    P.kf = pl.tbl_g_words ? t->dev.g_len : pl.k;
    P.Bt = pl.k ? t->dev.B[pl.k] : nullptr;
    P.tbl_b_words = pl.tbl_b_words;
    P.tbl_words = pl.tbl_words;
    P.tbl_c_words = pl.tbl_c_words;
    P.tbl_e_words = pl.tbl_e_words;
    P.rep_log2 = pl.rep_log2;
    P.dense_rows = pl.dense_rows;
    P.wait_limit_ns = opts && opts->test_wait_limit_us ? (uint64_t)opts->test_wait_limit_us * 1000
                                                       : WAIT_LIMIT_NS;
    P.withhold_unit = opts && opts->test_withhold_slice ? opts->test_withhold_slice - 1 : UNIT_NONE;
    if (pl.defer) {
        P.defer = (uint4 *)(W + L.defer);
        P.defer_cap = L.defer_cap;
        P.dbatch = (uint2 *)(W + L.dbatch);
        P.dbatch_cap = L.dbatch_cap;
    }
    const uint32_t nthreads = pl.queued ? pl.nw * 32 : NTHREADS;
    // units a CTA takes in one round: the register-staged kernel's warps
    // take two slices each
    const uint32_t units_per_cta = pl.queued ? (reg ? 2 * pl.nw : pl.nw) : 1;

    // header, and for the queued kernel the per-unit record and key counts
    // (the scan pass writes them only for units with kept survivors)
    cudaError_t e = cudaMemsetAsync(P.hdr, 0, pl.queued ? L.key_off : sizeof(WsHeader), st);
    const int nsm = sm_count();
    const uint32_t cps = opts && opts->ctas_per_sm ? opts->ctas_per_sm : 1;
    if (e == cudaSuccess && n_segments > 1 && P.n_tiles) {
        if (pl.queued) k_unitseg<<<nsm * 4, 256, 0, st>>>(P);
        else k_bounds<<<nsm * 2, 256, 0, st>>>(P);
        e = cudaGetLastError();
    }
    // persistent grid: one CTA per SM (fewer when there are few units)
    const uint64_t want = ((uint64_t)P.n_tiles + units_per_cta - 1) / units_per_cta;
    const uint32_t grid = (uint64_t)nsm * cps < want ? (uint32_t)nsm * cps : (uint32_t)want;
    if (e == cudaSuccess && opts && opts->ev_scan_begin)
        e = cudaEventRecord((cudaEvent_t)opts->ev_scan_begin, st);
    if (e == cudaSuccess && P.n_tiles) {
        int emit = 0;
        void *args[] = {&P, &emit};
        e = cudaLaunchKernel(pl.kernel, dim3(grid), dim3(nthreads), args, pl.smem, st);
    }
    if (e == cudaSuccess && P.n_tiles && pl.defer) {
        // the handed-over queues: prefix bitmap, counts and entries through
        // L2 (one bitmap copy)
        MatchParams P3 = P;
        P3.rep_log2 = 0;
        P3.tbl_e_words = 0;
        P3.tbl_m_words = 0;
        void *args[] = {&P3};
        e = cudaLaunchKernel(pl.kernel_res, dim3(nsm * RES_CTAS), dim3(RES_WARPS * 32), args, 0, st);
    }
    if (e == cudaSuccess && opts && opts->ev_scan_end)
        e = cudaEventRecord((cudaEvent_t)opts->ev_scan_end, st);
    if (e == cudaSuccess) {
        k_reduce<<<P.n_chunks ? P.n_chunks : 1, RT, 0, st>>>(P);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && P.n_tiles) {
        k_offsets<<<P.n_chunks, RT, 0, st>>>(P);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && opts && opts->ev_emit_begin)
        e = cudaEventRecord((cudaEvent_t)opts->ev_emit_begin, st);
    if (e == cudaSuccess && P.n_tiles) {
        int emit = 1;
        if (reg) {
            // the queued kernel re-scans the overflowing slices with its own
            // tables: one prefix-bitmap copy, entries through L2
            MatchParams P2 = P;
            P2.tbl_words = pl.e_tbl_words;
            P2.rep_log2 = 0;
            P2.tbl_e_words = 0;
            P2.tbl_m_words = pl.e_tbl_m_words;
            P2.tbl_g_words = 0;
            P2.g_rep = P2.g_fold = P2.g_hb = 0;
            P2.tbl_b_words = 0;
            P2.kf = pl.k;
            const uint64_t want_e = ((uint64_t)P.n_tiles + QW - 1) / QW;
            const uint32_t grid_e =
                (uint64_t)nsm * cps < want_e ? (uint32_t)nsm * cps : (uint32_t)want_e;
            void *args[] = {&P2, &emit};
            e = cudaLaunchKernel(pl.kernel_emit, dim3(grid_e), dim3(QW * 32), args, smem_emit, st);
        } else {
            void *args[] = {&P, &emit};
            e = cudaLaunchKernel(pl.kernel_emit, dim3(grid), dim3(nthreads), args, pl.smem, st);
        }
    }
    if (e == cudaSuccess && opts && opts->ev_emit_end)
        e = cudaEventRecord((cudaEvent_t)opts->ev_emit_end, st);
    if (e == cudaSuccess) {
        const uint64_t units = P.n_tiles ? P.n_tiles : 1;
        uint64_t blocks = (units + 255) / 256;
        const uint64_t maxb = (uint64_t)nsm * 8;
        if (blocks > maxb) blocks = maxb;
        k_expand<<<(uint32_t)blocks, 256, 0, st>>>(P);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return set_error(PFAC_ECUDA, "pfac_match: launch failed: %s", cudaGetErrorString(e));
    return PFAC_OK;
}

extern "C" int pfac_match(const pfac_table *t, const uint8_t *d_input, uint64_t n_bytes,
                          const uint64_t *d_seg_offsets, uint32_t n_segments, uint64_t *d_out_keys,
                          uint64_t out_capacity, uint64_t *n_out, const pfac_match_opts *opts,
                          void *cuda_stream) {
    clear_error();
    if (!t || !n_out) return set_error(PFAC_EINVAL, "pfac_match: NULL argument");
    if (!t->d_blob) return set_error(PFAC_EINVAL, "pfac_match: table was built host-only");
    int drc = check_table_device(t, cuda_stream, "pfac_match");
    if (drc) return drc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    uint64_t ws_bytes = 0;
    int rc0 = pfac_workspace_bytes(t, n_bytes, n_segments, opts, &ws_bytes);
    if (rc0) return rc0;
    void *ws = nullptr, *small = nullptr;
    cudaError_t e = cudaMallocAsync(&ws, ws_bytes, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&small, 256, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (ws) cudaFreeAsync(ws, st);
        return set_error(e == cudaErrorMemoryAllocation ? PFAC_ENOMEM : PFAC_ECUDA,
                         "pfac_match: workspace allocation: %s", cudaGetErrorString(e));
    }
    uint64_t *d_cnt = (uint64_t *)small;
    int32_t *d_st = (int32_t *)((uint8_t *)small + 128);
    int rc = pfac_match_async(t, d_input, n_bytes, d_seg_offsets, n_segments, d_out_keys,
                              out_capacity, d_cnt, d_st, ws, ws_bytes, opts, cuda_stream);
    struct {
        uint64_t cnt;
        int32_t st;
    } h{0, 0};
    if (rc == PFAC_OK) {
        e = cudaMemcpyAsync(&h.cnt, d_cnt, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h.st, d_st, 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = set_error(PFAC_ECUDA, "pfac_match: %s", cudaGetErrorString(e));
    }
    cudaFreeAsync(ws, st);
    cudaFreeAsync(small, st);
    if (rc) return rc;
    *n_out = h.cnt;
    if (h.st != PFAC_OK)
        return set_error(h.st, "pfac_match: device reported %s", pfac_status_str(h.st));
    if (h.cnt > out_capacity)
        return set_error(PFAC_ENOSPC, "pfac_match: %llu matches, capacity %llu",
                         (unsigned long long)h.cnt, (unsigned long long)out_capacity);
    return PFAC_OK;
}

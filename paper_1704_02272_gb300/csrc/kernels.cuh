// Device code shared by the matcher's kernels (sm_103a), and the tile-
// synchronous scan kernel used for the uncompressed state-transition table.
//
// k_scan (uncompressed table): a persistent grid, one CTA per SM.  Warp 16 is
// the producer: one lane streams 8 KiB tiles (plus a 16-byte halo) from HBM
// into a 4-stage shared-memory ring with cp.async.bulk, completion tracked by
// mbarriers.  Warps 0..15 consume: each thread owns 16 consecutive start
// positions and walks the table from the root (Section 2.3), the rows of the
// shallowest states held in shared memory.  A block scan gives each thread
// its slot; the tile's (position, fin) records go to a per-tile region of the
// workspace and the tile's match and key counts to per-unit counters.
//
// Ordering kernels (match.cu): k_reduce scans the per-unit key counts,
// k_offsets turns them into per-unit output offsets, k_expand writes the
// sorted keys of each unit from its records, and units whose records did not
// fit re-run the scan kernel in emit mode, which writes keys directly.  No
// kernel waits on another CTA; the only waits are mbarrier waits, each bounded
// by a wall-clock limit after which the kernel records PFAC_ETIMEOUT.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pfac.h"
#include "table.h"

namespace pfac {

constexpr int CW = 16;                  // consumer warps
constexpr int NCONS = CW * 32;          // consumer threads
constexpr int NTHREADS = NCONS + 32;    // plus one producer warp
constexpr int BPT = 16;                 // start positions per consumer thread
constexpr int TILE = NCONS * BPT;       // 8192 positions per tile
constexpr int HALO = 16;                // staged bytes past the tile (k - 1 <= 15)
constexpr int STAGES = 4;
constexpr int STAGE_IN = TILE + 128;    // bytes per input stage
constexpr int SEGW = 64;                // tile segment block: [count, <= 63 bounds]
constexpr int SEG_MAXB = SEGW - 1;
constexpr uint32_t SEG_OVF = 0xFFFFFFFFu;
constexpr int REC_CAP = TILE / 16;      // records kept per tile by the scan pass
constexpr int TABLE_SMEM_MAX = 128 * 1024;
constexpr uint64_t WAIT_LIMIT_NS = 4000000000ull;  // bounded waits: 4 s

constexpr int ST_BADSEG = 1, ST_TIMEOUT = 2, ST_DEVICE = 4;

// scan variants: prefix bitmap in shared memory with its entries in global
// memory (VAR_F) or in shared memory too (VAR_FE); uncompressed table (VAR_DENSE)
enum { VAR_F = 1, VAR_FE = 2, VAR_DENSE = 4 };
// kernel instances for merged tries (reduction step 2): VAR_F | VAR_MERGED;
// the others leave the merged-trie slow path out
constexpr int VAR_MERGED = 8;
// the resolver kernel's instances: VAR_F | VAR_RES (fewer walks per lane, so
// that more warps fit per SM)
constexpr int VAR_RES = 16;

struct WsHeader {
    int32_t status;
    uint32_t ovf_count;
    uint32_t done_reduce;
    uint32_t done_expand;
    uint32_t defer_entries;  // queue entries handed to the resolver kernel
    uint32_t defer_batches;  // and their batches
    uint32_t pad[10];
};

struct MatchParams {
    DevTable T;
    const uint8_t *in;
    uint64_t n;
    const uint64_t *seg;
    uint32_t n_seg;
    uint32_t n_tiles;     // ordering units of the scan kernel in use
    uint32_t unit_shift;  // log2 of the unit size in bytes
    uint32_t unit_cap;    // records kept per unit
    uint64_t *out;
    uint64_t cap;
    uint64_t *d_count;
    int32_t *d_status;
    // workspace
    WsHeader *hdr;
    uint32_t *tile_m;     // per unit: records kept, or more than unit_cap
    uint64_t *tile_k;     // per unit: keys
    uint64_t *key_off;    // per unit: first output slot
    uint64_t *chunk;      // n_chunks sums, then n_chunks offsets
    uint32_t n_chunks;
    uint32_t *ovf_list;
    uint64_t *recs;
    uint32_t *tile_bounds;  // tile-synchronous kernel: segment ends per tile
    uint32_t *unit_seg;     // queued kernel: first offset index after each unit start
    // scan configuration
    uint32_t k;           // prefix depth
    const uint32_t *F;    // prefix node of depth k: bitmap,
    const uint32_t *C;    //   block counts,
    const uint32_t *E;    //   entries
    const uint32_t *M;    //   child masks of the entries
    uint32_t tbl_words;   // shared-memory words: bitmap copies (or dense rows)
    uint32_t tbl_c_words;
    uint32_t tbl_e_words;
    uint32_t tbl_m_words; // child masks in shared memory (0 = not used)
    uint32_t c_shift;     // words per rank count of F_k (log2)
    uint32_t rep_log2;    // bitmap copies in shared memory (log2)
    uint32_t tbl_g_words; // gram filter in shared memory, all copies (0 = not used)
    uint32_t g_rep;       // gram filter copies (log2)
    uint32_t g_fold;      // gram filter words OR-ed together per shared word (log2)
    uint32_t g_hb;        // log2 of the shared gram filter's bits per copy
    uint32_t kf;          // symbols the first stage tests: k, or g with the gram filter
    const uint8_t *Bt;    // prefix bytes of depth k
    uint64_t starts_end;  // positions at or past it start no walk (<= n)
    uint64_t pos_base;    // added to every reported position
    uint32_t tbl_b_words; // prefix bytes in shared memory as the first stage (0 = not used)
    uint32_t dense_rows;  // dense layout: states whose rows live in shared memory
    // testing aids of the queued kernel: the bound of its waits, and a slice
    // whose copy is never issued (UNIT_NONE: none), so that the wait for it
    // runs out
    uint64_t wait_limit_ns;
    uint32_t withhold_unit;
    // queues of whole slices handed by the scan kernel to the resolver kernel
    // (register-staged plans): entries (16 bytes each) and batches {first, n}
    uint4 *defer;
    uint32_t defer_cap;
    uint32_t dbatch_cap;
    uint2 *dbatch;
};

constexpr uint32_t UNIT_NONE = 0xFFFFFFFFu;

// The bounds-checked build (compiled with PFAC_CHECKED, a separate library):
// the compressed-layout kernels pass every table, shared-memory, queue and
// input index through chk(), which, for an index at or past its bound,
// records ST_DEVICE in the call's status word (the call then reports
// PFAC_EDEVICE) and returns 0, always a valid index, so that no access leaves
// its array.  In the regular build chk() is the index itself.
#ifdef PFAC_CHECKED
constexpr bool CHECKED = true;
__device__ __forceinline__ uint64_t chk(const MatchParams &P, uint64_t i, uint64_t n) {
    if (i < n) return i;
    atomicOr(&P.hdr->status, ST_DEVICE);
    return 0;
}
#else
constexpr bool CHECKED = false;
__device__ __forceinline__ uint64_t chk(const MatchParams &, uint64_t i, uint64_t) { return i; }
#endif

// ------------------------------------------------------------ PTX helpers --

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase of `parity` to complete; gives up after limit_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  uint64_t limit_ns = WAIT_LIMIT_NS) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0;; it++) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63) == 63) {
            if (global_ns() - t0 > limit_ns) return false;
            __nanosleep(128);
        }
    }
}

// One bulk copy global -> this CTA's shared memory (no multicast); 16-byte
// aligned addresses, size a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void cons_bar() {
    asm volatile("bar.sync 1, %0;" ::"n"(NCONS) : "memory");
}

// Barrier over the consumer warps that also ANDs a predicate across them.
__device__ __forceinline__ bool cons_bar_and(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(NCONS)
        : "memory");
    return r != 0;
}

// ------------------------------------------------------------ outputs ------

__device__ __forceinline__ uint32_t fin_len(const uint32_t *__restrict__ pool, uint32_t f) {
    uint32_t l = f & FIN_LEN_ESC;
    return l == FIN_LEN_ESC ? __ldg(pool + (f >> FIN_LEN_BITS)) : l;
}

__device__ __forceinline__ const uint32_t *fin_ids(const uint32_t *__restrict__ pool, uint32_t f) {
    return pool + (f >> FIN_LEN_BITS) + (((f & FIN_LEN_ESC) == FIN_LEN_ESC) ? 1 : 0);
}

// fin_len / fin_ids of the table's pool with the list's words checked
// against the pool (a list past the pool reads as empty).
__device__ __forceinline__ uint32_t fin_len_c(const MatchParams &P, uint32_t f) {
    const uint32_t off = (uint32_t)chk(P, f >> FIN_LEN_BITS, P.T.pool_words);
    const bool esc = (f & FIN_LEN_ESC) == FIN_LEN_ESC;
    uint32_t l = esc ? __ldg(P.T.pool + off) : (f & FIN_LEN_ESC);
    if (CHECKED && (uint64_t)off + (esc ? 1u : 0u) + l > P.T.pool_words) {
        chk(P, 1, 0);
        l = 0;
    }
    return l;
}

__device__ __forceinline__ const uint32_t *fin_ids_c(const MatchParams &P, uint32_t f) {
    const uint32_t off = (uint32_t)chk(P, f >> FIN_LEN_BITS, P.T.pool_words);
    return P.T.pool + off + (((f & FIN_LEN_ESC) == FIN_LEN_ESC) ? 1 : 0);
}

// ------------------------------------------------------------ walks --------

// Uncompressed walk: state s, next-state table rows of sigma entries; rows of
// states below `nrows` are read from shared memory.
static __device__ __noinline__ uint32_t walk_dense(const uint32_t *__restrict__ stt,
                                            const uint32_t *__restrict__ dfin, uint32_t sigma,
                                            const uint32_t *srows, uint32_t nrows, uint32_t s,
                                            const uint8_t *sm, uint32_t staged,
                                            const uint8_t *__restrict__ g, uint32_t q,
                                            uint32_t lim) {
    while (q < lim) {
        const uint32_t c = q < staged ? (uint32_t)sm[q] : (uint32_t)__ldg(g + q);
        if (c >= sigma) break;
        const uint32_t nx = s < nrows ? srows[s * sigma + c] : __ldg(stt + (size_t)s * sigma + c);
        if (!nx) break;
        s = nx;
        q++;
    }
    return __ldg(dfin + s);
}

// ------------------------------------------------------------ packing ------

// Packs the 32 window bytes into a bit string of BPS bits per symbol (first
// symbol lowest); bs has BPS + 1 words, the last one zero.
template <int BPS>
__device__ __forceinline__ void pack_symbols(const uint32_t (&x)[8], uint32_t (&bs)[BPS + 1]) {
    if (BPS == 8) {
#pragma unroll
        for (int w = 0; w < 8; w++) bs[w] = x[w];
        bs[BPS] = 0;
    } else if (BPS == 2) {
        // four 2-bit symbols s0..s3 in the low bits of four bytes -> one byte
        // s0 | s1 << 2 | s2 << 4 | s3 << 6: the multiplier places copies of the
        // word at shifts 6, 12, 18, 24, so that bit 24 + 2i receives s_i and no
        // other partial product reaches bits 24..31 (checked for all 256
        // inputs); three byte permutes gather the four top bytes
        uint32_t b[8];
#pragma unroll
        for (int w = 0; w < 8; w++) b[w] = (x[w] & 0x03030303u) * 0x01041040u;
        bs[0] = __byte_perm(__byte_perm(b[0], b[1], 0x0073), __byte_perm(b[2], b[3], 0x0073),
                            0x5410);
        bs[1] = __byte_perm(__byte_perm(b[4], b[5], 0x0073), __byte_perm(b[6], b[7], 0x0073),
                            0x5410);
        bs[2] = 0;
    } else {
#pragma unroll
        for (int w = 0; w <= BPS; w++) bs[w] = 0;
#pragma unroll
        for (int i = 0; i < 32; i++) {
            const uint32_t s = (x[i >> 2] >> (8 * (i & 3))) & ((1u << BPS) - 1u);
            const int bit = BPS * i;
            bs[bit >> 5] |= s << (bit & 31);
            if ((bit & 31) + BPS > 32) bs[(bit >> 5) + 1] |= s >> (32 - (bit & 31));
        }
    }
}

// Bits [BPS*j, BPS*j + 32) of the packed string.
template <int BPS>
__device__ __forceinline__ uint32_t symbols_at(const uint32_t (&bs)[BPS + 1], int j) {
    const int bit = BPS * j;
    return __funnelshift_r(bs[bit >> 5], bs[(bit >> 5) + 1], bit & 31);
}

// ------------------------------------------------------------ tile pieces --

// First segment end strictly above relative position p (clipped to rem).
__device__ __forceinline__ uint32_t seg_limit(const uint32_t *segs, uint32_t p, uint32_t rem,
                                              const uint64_t *__restrict__ gseg, uint32_t n_seg,
                                              uint64_t tile_start) {
    if (n_seg <= 1) return rem;
    const uint32_t nb = segs[0];
    if (nb == SEG_OVF) {
        // more boundaries than the tile block holds: search the offsets
        const uint64_t ap = tile_start + p;
        uint32_t lo = 1, hi = n_seg;  // first index s in [1, n_seg] with o_s > ap
        while (lo < hi) {
            uint32_t mid = (lo + hi) >> 1;
            if (__ldg(gseg + mid) > ap) hi = mid; else lo = mid + 1;
        }
        const uint64_t e = __ldg(gseg + lo);
        const uint64_t r = e > tile_start ? e - tile_start : 0;
        return r < rem ? (uint32_t)r : rem;
    }
    uint32_t lo = 0, hi = nb;  // first entry > p among segs[1..nb]
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (segs[1 + mid] > p) hi = mid; else lo = mid + 1;
    }
    const uint32_t r = lo < nb ? segs[1 + lo] : rem;
    return r < rem ? r : rem;
}

// Walk results of one thread's 16 positions (uncompressed layout).
__device__ __forceinline__ void thread_positions_dense(const MatchParams &P, const uint8_t *sin,
                                                       uint32_t staged, uint32_t valid,
                                                       uint32_t rem, const uint32_t *segs,
                                                       uint64_t tile_start,
                                                       const uint8_t *__restrict__ g,
                                                       const uint32_t *srows, uint32_t tid,
                                                       uint32_t (&fr)[BPT]) {
    const uint32_t p0 = tid * BPT;
    const uint32_t sigma = P.T.sigma;
#pragma unroll
    for (int j = 0; j < BPT; j++) fr[j] = 0;
    if (p0 >= valid) return;
    const uint32_t lim = seg_limit(segs, p0, rem, P.seg, P.n_seg, tile_start);
    const uint32_t span = p0 + BPT;
    if (span <= lim && span <= staged && span <= valid) {
        const uint4 a = *reinterpret_cast<const uint4 *>(sin + p0);
        const uint32_t x[4] = {a.x, a.y, a.z, a.w};
        uint32_t s1[BPT];
        uint32_t surv = 0;
#pragma unroll
        for (int j = 0; j < BPT; j++) {
            const uint32_t c = (x[j >> 2] >> (8 * (j & 3))) & 0xFFu;
            s1[j] = c < sigma ? srows[c] : 0u;  // root row is row 0 in shared memory
            surv |= (s1[j] != 0 ? 1u : 0u) << j;
        }
        if (surv) {
#pragma unroll
            for (int j = 0; j < BPT; j++)
                if ((surv >> j) & 1u)
                    fr[j] = walk_dense(P.T.stt, P.T.dfin, sigma, srows, P.dense_rows, s1[j], sin,
                                       staged, g, p0 + j + 1, lim);
        }
        return;
    }
#pragma unroll 1
    for (int j = 0; j < BPT; j++) {
        const uint32_t p = p0 + j;
        if (p >= valid) break;
        const uint32_t lj = seg_limit(segs, p, rem, P.seg, P.n_seg, tile_start);
        const uint32_t f = walk_dense(P.T.stt, P.T.dfin, sigma, srows, P.dense_rows, 0u, sin,
                                      staged, g, p, lj);
#pragma unroll
        for (int i = 0; i < BPT; i++)
            if (i == j) fr[i] = f;
    }
}

// Exclusive scan over the consumer threads; returns the prefix, sets total.
__device__ __forceinline__ uint64_t cons_scan(uint64_t v, uint64_t *wt, uint64_t &total,
                                              uint32_t tid) {
    const uint32_t lane = tid & 31, w = tid >> 5;
    uint64_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t nb = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= (uint32_t)o) inc += nb;
    }
    if (lane == 31) wt[w] = inc;
    cons_bar();
    if (w == 0) {
        uint64_t t = lane < CW ? wt[lane] : 0;
        uint64_t ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t nb = __shfl_up_sync(0xFFFFFFFFu, ti, o);
            if (lane >= (uint32_t)o) ti += nb;
        }
        if (lane < CW) wt[lane] = ti - t;
        if (lane == CW - 1) wt[CW] = ti;
    }
    cons_bar();
    total = wt[CW];
    return wt[w] + inc - v;
}

// ------------------------------------------------------------ scan kernel --

#ifdef PFAC_DEFINE_DENSE_KERNEL
// Scan kernel of the uncompressed table.
// emit == 0: scan every tile, keep records, count keys.
// emit == 1: re-run the tiles listed in ovf_list and write their keys.
__global__ void __launch_bounds__(NTHREADS, 1) k_scan_dense(const MatchParams P, const int emit) {
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t tbl_bytes = (P.tbl_words * 4u + 127u) & ~127u;
    uint32_t *stbl = reinterpret_cast<uint32_t *>(smem);
    uint8_t *st_in = smem + tbl_bytes;
    uint32_t *st_seg = reinterpret_cast<uint32_t *>(st_in + STAGES * STAGE_IN);
    uint64_t *full = reinterpret_cast<uint64_t *>(st_seg + STAGES * SEGW);
    uint64_t *empty = full + STAGES;
    int32_t *st_tile = reinterpret_cast<int32_t *>(empty + STAGES);
    uint64_t *wt = reinterpret_cast<uint64_t *>(st_tile + 2 * STAGES);

    const uint32_t tid = threadIdx.x;
    const uint32_t n_work = emit ? *(volatile uint32_t *)&P.hdr->ovf_count : P.n_tiles;
    if (blockIdx.x >= n_work) return;

    if (tid == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], CW);
        }
        fence_barrier_init();
    }
    __syncthreads();

    if (tid >= NCONS) {
        // ---------------- producer warp ----------------
        if (tid == NCONS) {
            uint32_t issued = 0;
            bool timed_out = false;
            for (uint32_t i = 0;; i++) {
                const int s = i % STAGES;
                if (i >= STAGES && !mbar_wait_bounded(&empty[s], ((i / STAGES) - 1) & 1)) {
                    // the consumers stopped releasing stages; they give up on
                    // their own bounded waits
                    atomicOr(&P.hdr->status, ST_TIMEOUT);
                    timed_out = true;
                    break;
                }
                const uint32_t wi = blockIdx.x + i * gridDim.x;
                if (wi >= n_work) {
                    st_tile[s] = -1;
                    mbar_arrive(&full[s]);
                    break;
                }
                const uint32_t t = emit ? P.ovf_list[wi] : wi;
                st_tile[s] = (int32_t)t;
                const uint64_t start = (uint64_t)t * TILE;
                const uint64_t avail = P.n - start;
                const uint32_t bytes = avail < (uint64_t)(TILE + HALO) ? (uint32_t)avail : TILE + HALO;
                const uint32_t nb = bytes & ~15u;
                const uint32_t tx = nb + (P.n_seg > 1 ? SEGW * 4 : 0);
                mbar_arrive_expect_tx(&full[s], tx);
                if (nb) bulk_g2s(st_in + s * STAGE_IN, P.in + start, nb, &full[s]);
                if (P.n_seg > 1)
                    bulk_g2s(st_seg + s * SEGW, P.tile_bounds + (size_t)t * SEGW, SEGW * 4,
                             &full[s]);
                issued = i + 1;
            }
            // On the normal path every issued copy is waited for by the
            // consumers before the CTA can exit.  After a timeout, wait
            // (bounded) for the copies that may still be in flight.
            if (timed_out)
                for (uint32_t i = issued > STAGES ? issued - STAGES : 0; i < issued; i++)
                    mbar_wait_bounded(&full[i % STAGES], (i / STAGES) & 1);
        }
        return;
    }

    // ---------------- consumer warps ----------------
    for (uint32_t i = tid; i < P.tbl_words; i += NCONS) stbl[i] = __ldg(P.T.stt + i);
    cons_bar();

    const uint32_t lane = tid & 31;
    for (uint32_t i = 0;; i++) {
        const int s = i % STAGES;
        const bool ok = cons_bar_and(mbar_wait_bounded(&full[s], (i / STAGES) & 1));
        if (!ok) {
            if (tid == 0) atomicOr(&P.hdr->status, ST_TIMEOUT);
            break;
        }
        const int32_t t = st_tile[s];
        if (t < 0) break;
        const uint64_t tile_start = (uint64_t)t * TILE;
        const uint64_t remain = P.n - tile_start;
        const uint32_t rem = remain < 0xFFFFFFF0ull ? (uint32_t)remain : 0xFFFFFFF0u;
        uint32_t valid = rem < (uint32_t)TILE ? rem : (uint32_t)TILE;
        {
            const uint64_t sl = P.starts_end > tile_start ? P.starts_end - tile_start : 0;
            if (sl < valid) valid = (uint32_t)sl;
        }
        const uint32_t staged = (rem < (uint32_t)(TILE + HALO) ? rem : (uint32_t)(TILE + HALO)) & ~15u;
        const uint8_t *sin = st_in + s * STAGE_IN;
        const uint32_t *segs = st_seg + s * SEGW;
        const uint8_t *g = P.in + tile_start;

        uint32_t fr[BPT];
        thread_positions_dense(P, sin, staged, valid, rem, segs, tile_start, g, stbl, tid, fr);
        // the stage is no longer read: hand it back to the producer
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);

        uint32_t nm = 0;
        uint64_t nk = 0;
#pragma unroll
        for (int j = 0; j < BPT; j++) {
            if (fr[j]) {
                nm++;
                nk += fin_len_c(P, fr[j]);
            }
        }
        uint64_t total;
        const uint64_t excl = cons_scan((nk << 16) | nm, wt, total, tid);
        const uint32_t m_t = (uint32_t)(total & 0xFFFFu);
        const uint64_t k_t = total >> 16;
        const uint32_t p0 = tid * BPT;
        if (!emit) {
            if (m_t <= (uint32_t)REC_CAP) {
                uint64_t *rr = P.recs + (size_t)t * REC_CAP + (excl & 0xFFFFu);
#pragma unroll
                for (int j = 0; j < BPT; j++)
                    if (fr[j]) *rr++ = ((uint64_t)(p0 + j) << 32) | fr[j];
            }
            if (tid == 0) {
                P.tile_m[t] = m_t;
                P.tile_k[t] = k_t;
                if (m_t > (uint32_t)REC_CAP) P.ovf_list[atomicAdd(&P.hdr->ovf_count, 1u)] = t;
            }
        } else if (nm) {
            uint64_t o = P.key_off[t] + (excl >> 16);
#pragma unroll 1
            for (int j = 0; j < BPT; j++) {
                const uint32_t f = fr[j];
                if (!f) continue;
                const uint32_t L = fin_len_c(P, f);
                const uint32_t *ids = fin_ids_c(P, f);
                const uint64_t pk = (P.pos_base + tile_start + p0 + j) << PFAC_ID_BITS;
                for (uint32_t e = 0; e < L; e++, o++)
                    if (o < P.cap) P.out[o] = pk | __ldg(ids + e);
            }
        }
    }
}

#endif  // PFAC_DEFINE_DENSE_KERNEL

}  // namespace pfac

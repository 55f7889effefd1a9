// Queued scan kernel for the compressed layout (Section 2.3 walk over the
// Section 3.1 records), built so that no warp waits for another.
//
// * Work unit: a 512-byte slice of the input.  Slice g goes to global warp
//   g mod (warps in the grid); every warp streams its own slices with
//   cp.async.bulk into a private 4-stage ring of 528-byte stages (slice plus
//   a 16-byte halo), each stage with its own mbarrier.
// * Filter: each lane owns 16 start positions of the slice.  For each it
//   forms the index of the next k symbols and tests the depth-k prefix
//   bitmap F_k held in shared memory (replicated over bank groups so a
//   warp's 32 random lookups conflict little).  Positions whose k-symbol
//   window is not available (segment end, input end, symbol outside the
//   packed range) become "root" survivors that walk from the root.
// * Survivors go to a per-warp queue in shared memory.  When it is nearly
//   full the warp resolves it in one batch: four queue entries per lane, all
//   advanced in lockstep, so each lane keeps several independent loads in
//   flight.  Resolution ranks the prefix index in F_k (block counts C_k plus
//   popcounts, Eq. 1 applied to the prefix level) to read its entry E_k (the
//   state at depth k or the output of a walk that stopped earlier), then walks
//   the records through L2 one level per round.
// * Output: per slice, the survivors' (position, fin) records in position
//   order plus the slice's key count; slices with more survivors than their
//   record space are resolved immediately in quarters (counting only) and
//   re-run by the emit pass, which writes their keys directly.
#pragma once
#include "kernels.cuh"

namespace pfac {

constexpr int QW = 16;                   // warps per CTA
constexpr int QTHREADS = QW * 32;
constexpr int QBPT = 16;                 // start positions per lane per slice
constexpr int SLICE = 32 * QBPT;         // 512 start positions per slice
constexpr int SLICE_SHIFT = 9;
constexpr int QRING = 4;                 // stages per warp ring
constexpr int QSTAGE = SLICE + 16;       // bytes per stage: slice plus halo
constexpr int SCAP = 32;                 // match records kept per slice by the scan pass
constexpr int QCAP = 128;                // queue entries per warp (and most survivors
                                         // of one slice queued at once)
constexpr int QU = QCAP / 32;            // queue entries per lane per batch
constexpr uint32_t ROOT_X = 0xFFFFFFFFu; // queue entry: walk from the root
constexpr uint32_t UNIT_OVF = 0xFFFFFFFFu;
constexpr uint32_t LIM_MAX = 0xFFFFFFF0u;

struct QEntry {
    uint32_t unit;
    uint32_t pos;   // position in the slice | slot << 10 | survivors of the slice << 18
    uint32_t x;     // prefix index, or ROOT_X
    uint32_t lim;   // walk limit relative to the slice start
};

struct WarpArea {
    uint8_t ring[QRING][QSTAGE];
    QEntry q[QCAP];
    uint64_t bar[QRING];
};

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Rank of prefix index x among the set bits of F_k (Eq. 1 on the prefix
// level): block count plus popcounts of the preceding words of its block.
__device__ __forceinline__ uint32_t prefix_rank(const uint32_t *Fs, uint32_t rep,
                                                const uint32_t *Cs, uint32_t x) {
    const uint32_t w = x >> 5, b0 = (x >> 8) << 3;
    uint32_t r = Cs[x >> 8];
    for (uint32_t i = b0; i < w; i++) r += __popc(Fs[i << rep]);
    return r + __popc(Fs[w << rep] & ((1u << (x & 31)) - 1u));
}

// One batch: resolve up to QCAP queue entries (entry e handled by lane e % 32,
// slot e / 32).  Each entry ends with the fin of the state its walk stops at.
template <int W, int VAR>
__device__ __forceinline__ void resolve_batch(const MatchParams &P, const QEntry *q, uint32_t n,
                                              const uint32_t *Fs, const uint32_t *Cs,
                                              const uint32_t *Es, uint32_t lane,
                                              uint32_t (&fin)[QU], uint32_t (&pos)[QU],
                                              uint32_t (&unit)[QU]) {
    constexpr int RW = rec_words(W);
    const uint32_t sigma = P.T.sigma, k = P.k, rep = P.rep_log2;
    const uint32_t *__restrict__ rec = P.T.rec;
    uint32_t st[QU], qq[QU], lim[QU], ev[QU];
    bool walk[QU];
    // ---- phase A: prefix entries (independent loads for all entries)
#pragma unroll
    for (int u = 0; u < QU; u++) {
        const uint32_t e = lane + 32u * u;
        fin[u] = 0;
        walk[u] = false;
        st[u] = 0;
        qq[u] = 0;
        lim[u] = 0;
        ev[u] = 0;
        pos[u] = 0;
        unit[u] = 0xFFFFFFFFu;
        if (e < n) {
            const QEntry en = q[e];
            unit[u] = en.unit;
            pos[u] = en.pos;
            lim[u] = en.lim;
            const uint32_t p = en.pos & 0x3FFu;
            if (en.x == ROOT_X) {
                walk[u] = true;
                st[u] = 0;
                qq[u] = p;
            } else {
                const uint32_t r = prefix_rank(Fs, rep, Cs, en.x);
                ev[u] = VAR == VAR_FE ? Es[r] : __ldg(P.E + r);
                qq[u] = p + k;
            }
        }
    }
#pragma unroll
    for (int u = 0; u < QU; u++) {
        if (unit[u] != 0xFFFFFFFFu && !walk[u]) {
            if (ev[u] & D_CONT) {
                walk[u] = true;
                st[u] = ev[u] & D_VAL_MASK;
            } else {
                fin[u] = ev[u];
            }
        }
    }
    // ---- phase B: walk rounds, one trie level per round for every entry
    uint32_t leaf_at[QU];
#pragma unroll
    for (int u = 0; u < QU; u++) leaf_at[u] = 0xFFFFFFFFu;
    for (;;) {
        bool any = false;
#pragma unroll
        for (int u = 0; u < QU; u++) any |= walk[u];
        if (!__any_sync(0xFFFFFFFFu, any)) break;
        uint32_t c[QU], f1[QU], m0[QU], m1[QU];
        uint4 b0[QU], b1[QU];
#pragma unroll
        for (int u = 0; u < QU; u++) {
            if (walk[u]) {
                const uint64_t ab = ((uint64_t)unit[u] << SLICE_SHIFT) + qq[u];
                c[u] = qq[u] < lim[u] ? (uint32_t)__ldg(P.in + ab) : 0x100u;
                const uint32_t *R = rec + (size_t)st[u] * RW;
                if (W == 1) {
                    const uint2 v = __ldg(reinterpret_cast<const uint2 *>(R));
                    b0[u].x = v.x;
                    m0[u] = v.y;
                    f1[u] = __ldg(P.T.fin + st[u]);
                } else if (W == 2) {
                    b0[u] = __ldg(reinterpret_cast<const uint4 *>(R));
                    m0[u] = b0[u].z;
                    f1[u] = b0[u].w;
                } else {
                    b0[u] = __ldg(reinterpret_cast<const uint4 *>(R));
                    b1[u] = __ldg(reinterpret_cast<const uint4 *>(R + 4));
                    const uint2 mf = __ldg(reinterpret_cast<const uint2 *>(R + 8));
                    const uint2 cu = __ldg(reinterpret_cast<const uint2 *>(R + 10));
                    m0[u] = mf.x;
                    f1[u] = mf.y;
                    m1[u] = (c[u] & 0x80u) ? cu.y : cu.x;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < QU; u++) {
            if (!walk[u]) continue;
            const uint32_t cc = c[u];
            uint32_t word = 0, below = 0;
            if (cc < sigma) {
                if (W == 1) {
                    word = b0[u].x;
                } else if (W == 2) {
                    word = cc < 32 ? b0[u].x : b0[u].y;
                    below = cc < 32 ? 0u : (uint32_t)__popc(b0[u].x);
                } else {
                    const uint32_t wi = cc >> 5;
                    const uint4 h = wi < 4 ? b0[u] : b1[u];
                    const uint32_t wj = wi & 3;
                    word = wj == 0 ? h.x : (wj == 1 ? h.y : (wj == 2 ? h.z : h.w));
                    below = (m1[u] >> (8 * wj)) & 0xFFu;
                }
            }
            const uint32_t bit = cc & 31;
            if (cc >= sigma || !((word >> bit) & 1u)) {
                fin[u] = f1[u];
                walk[u] = false;
                continue;
            }
            const uint32_t rank = below + (uint32_t)__popc(word & ((1u << bit) - 1u));
            const uint32_t base = m0[u] & META_BASE_MASK;
            if (m0[u] & META_ALL_LEAF) {
                leaf_at[u] = base + rank;
                walk[u] = false;
                continue;
            }
            st[u] = base + rank;
            qq[u]++;
        }
    }
#pragma unroll
    for (int u = 0; u < QU; u++)
        if (leaf_at[u] != 0xFFFFFFFFu) fin[u] = __ldg(P.T.leaf_fin + leaf_at[u]);
}

// Filter of one slice by one warp.  Fills the survivor masks of the lane's
// 16 positions and their walk limits (relative to the slice start).
template <int BPS>
__device__ __forceinline__ void filter_slice(const MatchParams &P, const uint8_t *sb,
                                             uint32_t staged, uint32_t valid, uint32_t rem,
                                             uint32_t lima, uint32_t limb, bool general_lims,
                                             const uint64_t *__restrict__ gseg, uint64_t ustart,
                                             const uint32_t *Fs, uint32_t lane, uint32_t &surv,
                                             uint32_t &rootm) {
    const uint32_t p0 = lane * QBPT;
    const uint32_t k = P.k, rep = P.rep_log2;
    surv = 0;
    rootm = 0;
    if (p0 >= valid) return;
    const uint4 a = *reinterpret_cast<const uint4 *>(sb + p0);
    const uint4 b = *reinterpret_cast<const uint4 *>(sb + p0 + 16);
    const uint32_t x[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    uint32_t bs[BPS + 1];
    pack_symbols<BPS>(x, bs);
    const uint32_t kmask = (1u << (BPS * k)) - 1u;
    const uint32_t copy = lane & ((1u << rep) - 1u);
#pragma unroll
    for (int j = 0; j < QBPT; j++) {
        const uint32_t idx = symbols_at<BPS>(bs, j) & kmask;
        const uint32_t w = Fs[((idx >> 5) << rep) | copy];
        surv |= ((w >> (idx & 31)) & 1u) << j;
    }
    // positions whose k-symbol window is available in this segment and stage
    const uint32_t lim0 = lima < staged ? lima : staged;
    uint32_t badb = 0;  // bytes of the window outside the packed symbol range
    if (BPS < 8) {
        const uint32_t hm = 0x01010101u * ((0xFFu << BPS) & 0xFFu);
        uint32_t any = 0;
#pragma unroll
        for (int w = 0; w < 8; w++) any |= x[w] & hm;
        if (any) {
#pragma unroll
            for (int i = 0; i < 32; i++)
                if ((x[i >> 2] >> (8 * (i & 3))) & ((0xFFu << BPS) & 0xFFu)) badb |= 1u << i;
        }
    }
    const uint32_t kwin = (k >= 32) ? 0xFFFFFFFFu : ((1u << k) - 1u);
    // every position's window is available (the window limits are exact
    // only when the slice's segment ends fit the lane's window)
    if (!general_lims && p0 + QBPT - 1 + k <= lim0 && badb == 0) return;
    uint32_t fv = 0, ex = 0;
#pragma unroll 1
    for (int j = 0; j < QBPT; j++) {
        const uint32_t p = p0 + j;
        if (p >= valid) break;
        uint32_t lj;
        if (!general_lims) {
            lj = p < lima ? lima : limb;
        } else {
            uint32_t lo = 1, hi = P.n_seg;
            const uint64_t ap = ustart + p;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (__ldg(gseg + mid) > ap) hi = mid; else lo = mid + 1;
            }
            const uint64_t e = __ldg(gseg + lo);
            const uint64_t r = e > ustart ? e - ustart : 0;
            lj = r < rem ? (uint32_t)r : rem;
        }
        if (lj > p) ex |= 1u << j;
        const uint32_t lw = lj < staged ? lj : staged;
        if (p + k <= lw && ((badb >> j) & kwin) == 0) fv |= 1u << j;
    }
    surv &= fv;
    rootm = ex & ~fv;
}

// Walk limit of position p (relative), for queue entries.
__device__ __forceinline__ uint32_t lim_of(const MatchParams &P, uint32_t p, uint32_t lima,
                                           uint32_t limb, bool general_lims, uint64_t ustart,
                                           uint32_t rem) {
    if (!general_lims) return p < lima ? lima : limb;
    uint32_t lo = 1, hi = P.n_seg;
    const uint64_t ap = ustart + p;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(P.seg + mid) > ap) hi = mid; else lo = mid + 1;
    }
    const uint64_t e = __ldg(P.seg + lo);
    const uint64_t r = e > ustart ? e - ustart : 0;
    return r < rem ? (uint32_t)r : rem;
}

// Prefix index of position p from the staged bytes (survivors only).
template <int BPS>
__device__ __forceinline__ uint32_t index_at(const uint8_t *sb, uint32_t p, uint32_t k) {
    uint32_t x = 0;
    for (uint32_t i = 0; i < k; i++) x |= ((uint32_t)sb[p + i] & ((1u << BPS) - 1u)) << (BPS * i);
    return x;
}

// Appends the survivors of lanes whose bit is set in `lanes` to the queue at
// qn, in position order.  Returns the number appended (warp-uniform).
template <int BPS>
__device__ __forceinline__ uint32_t append_survivors(const MatchParams &P, QEntry *q, uint32_t qn,
                                                     uint32_t surv, uint32_t rootm, uint32_t lanes,
                                                     const uint8_t *sb, uint32_t unit,
                                                     uint32_t lima, uint32_t limb,
                                                     bool general_lims, uint64_t ustart,
                                                     uint32_t rem, uint32_t lane,
                                                     uint32_t slot_base) {
    uint32_t m = ((lanes >> lane) & 1u) ? (surv | rootm) : 0u;
    const uint32_t c = __popc(m);
    uint32_t inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t nb = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= (uint32_t)o) inc += nb;
    }
    const uint32_t tot = __shfl_sync(0xFFFFFFFFu, inc, 31);
    uint32_t o = inc - c;
    const uint32_t p0 = lane * QBPT;
    while (m) {
        const uint32_t j = __ffs(m) - 1;
        m &= m - 1;
        const uint32_t p = p0 + j;
        QEntry en;
        en.unit = unit;
        en.pos = p | ((slot_base + o) << 10) | (tot << 18);
        en.x = ((rootm >> j) & 1u) ? ROOT_X : index_at<BPS>(sb, p, P.k);
        en.lim = lim_of(P, p, lima, limb, general_lims, ustart, rem);
        q[qn + o] = en;
        o++;
    }
    __syncwarp();
    return tot;
}

// Record-mode flush: resolve the queue, then keep a record (position, fin)
// for each matched survivor, ranked among its slice's matched survivors (the
// slice's entries are contiguous in the queue and resolve in one batch).
// The last entry of each slice publishes the slice's record count; slices
// with more matches than their record space go to the emit pass.
template <int W, int VAR>
__device__ __forceinline__ void flush_records(const MatchParams &P, QEntry *q, uint32_t n,
                                              const uint32_t *Fs, const uint32_t *Cs,
                                              const uint32_t *Es, uint32_t lane) {
    if (n == 0) return;
    uint32_t fin[QU], pos[QU], unit[QU];
    resolve_batch<W, VAR>(P, q, n, Fs, Cs, Es, lane, fin, pos, unit);
    // exclusive count of matched entries before each entry of the batch
    uint32_t pre[QU], carry = 0;
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int u = 0; u < QU; u++) {
        const uint32_t b = __ballot_sync(0xFFFFFFFFu, fin[u] != 0);
        pre[u] = carry + __popc(b & lt);
        carry += __popc(b);
    }
#pragma unroll
    for (int u = 0; u < QU; u++)
        if (unit[u] != 0xFFFFFFFFu) q[lane + 32u * u].x = pre[u];
    __syncwarp();
#pragma unroll
    for (int u = 0; u < QU; u++) {
        if (unit[u] == 0xFFFFFFFFu) continue;
        const uint32_t e = lane + 32u * u;
        const uint32_t p = pos[u] & 0x3FFu, slot = (pos[u] >> 10) & 0xFFu, cnt = pos[u] >> 18;
        const uint32_t base = q[e - slot].x;
        const uint32_t rank = pre[u] - base;
        if (fin[u]) {
            if (rank < (uint32_t)SCAP)
                P.recs[(size_t)unit[u] * SCAP + rank] = ((uint64_t)p << 32) | fin[u];
            atomicAdd((unsigned long long *)(P.tile_k + unit[u]),
                      (unsigned long long)fin_len(P.T.pool, fin[u]));
        }
        if (slot + 1 == cnt) {
            const uint32_t m = rank + (fin[u] ? 1u : 0u);
            if (m > (uint32_t)SCAP) {
                P.tile_m[unit[u]] = UNIT_OVF;
                P.ovf_list[atomicAdd(&P.hdr->ovf_count, 1u)] = unit[u];
            } else {
                P.tile_m[unit[u]] = m;
            }
        }
    }
    __syncwarp();
}

// Resolves every survivor of one slice in quarters of 8 lanes (at most 128
// entries each).  emit == 0: returns the slice's key count.  emit == 1:
// writes the slice's keys at key_off[unit] and returns the count.
template <int W, int BPS, int VAR>
__device__ __forceinline__ uint64_t resolve_slice(const MatchParams &P, QEntry *q, uint32_t surv,
                                                  uint32_t rootm, const uint8_t *sb,
                                                  uint32_t unitid, uint32_t lima, uint32_t limb,
                                                  bool general_lims, uint64_t ustart,
                                                  uint32_t rem, const uint32_t *Fs,
                                                  const uint32_t *Cs, const uint32_t *Es,
                                                  uint32_t lane, bool emit) {
    uint64_t keys = 0;
    const uint64_t obase = emit ? P.key_off[unitid] : 0;
    for (int qt = 0; qt < 4; qt++) {
        const uint32_t n = append_survivors<BPS>(P, q, 0, surv, rootm, 0xFFu << (8 * qt), sb,
                                                 unitid, lima, limb, general_lims, ustart, rem,
                                                 lane, 0);
        if (n == 0) continue;
        uint32_t fin[QU], pos[QU], unit[QU];
        resolve_batch<W, VAR>(P, q, n, Fs, Cs, Es, lane, fin, pos, unit);
#pragma unroll
        for (int u = 0; u < QU; u++) {
            const uint32_t L = fin[u] ? fin_len(P.T.pool, fin[u]) : 0u;
            uint32_t inc = L;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t nb = __shfl_up_sync(0xFFFFFFFFu, inc, o);
                if (lane >= (uint32_t)o) inc += nb;
            }
            const uint32_t tot = __shfl_sync(0xFFFFFFFFu, inc, 31);
            if (emit && L) {
                const uint32_t *ids = fin_ids(P.T.pool, fin[u]);
                const uint64_t pk = (ustart + (pos[u] & 0x3FFu)) << PFAC_ID_BITS;
                uint64_t o = obase + keys + inc - L;
                for (uint32_t e = 0; e < L; e++, o++)
                    if (o < P.cap) P.out[o] = pk | __ldg(ids + e);
            }
            keys += tot;
        }
        __syncwarp();
    }
    return keys;
}

template <int W, int BPS, int VAR>
__global__ void __launch_bounds__(QTHREADS, 1) k_scanq(const MatchParams P, const int emit) {
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t n_units = emit ? *(volatile uint32_t *)&P.hdr->ovf_count : P.n_tiles;
    const uint32_t gw = blockIdx.x * QW + warp, gstride = gridDim.x * QW;
    if (blockIdx.x * QW >= n_units) return;  // the whole CTA has no unit

    uint32_t *Fs = reinterpret_cast<uint32_t *>(smem);
    uint32_t *Cs = Fs + P.tbl_words;
    uint32_t *Es = Cs + P.tbl_c_words;
    WarpArea *areas = reinterpret_cast<WarpArea *>(
        smem + ((((size_t)P.tbl_words + P.tbl_c_words + P.tbl_e_words) * 4 + 127) & ~(size_t)127));
    {
        const uint32_t rep = P.rep_log2;
        for (uint32_t i = threadIdx.x; i < P.tbl_words; i += QTHREADS) Fs[i] = __ldg(P.F + (i >> rep));
        for (uint32_t i = threadIdx.x; i < P.tbl_c_words; i += QTHREADS) Cs[i] = __ldg(P.C + i);
        if (VAR == VAR_FE)
            for (uint32_t i = threadIdx.x; i < P.tbl_e_words; i += QTHREADS) Es[i] = __ldg(P.E + i);
    }
    WarpArea &A = areas[warp];
    if (lane == 0) {
        for (int s = 0; s < QRING; s++) mbar_init(&A.bar[s], 1);
        fence_barrier_init();
    }
    __syncthreads();

    auto unit_of = [&](uint32_t i) -> uint32_t {
        const uint32_t wi = gw + i * gstride;
        return emit ? P.ovf_list[wi] : wi;
    };
    auto issue = [&](uint32_t i) {
        // lane 0 only: stage i % QRING <- slice of the warp's i-th unit
        const uint32_t wi = gw + i * gstride;
        if (wi >= n_units) return;
        const uint32_t u = unit_of(i);
        const uint64_t start = (uint64_t)u << SLICE_SHIFT;
        const uint64_t avail = P.n - start;
        const uint32_t bytes = (avail < (uint64_t)QSTAGE ? (uint32_t)avail : (uint32_t)QSTAGE) & ~15u;
        uint64_t *bar = &A.bar[i % QRING];
        mbar_arrive_expect_tx(bar, bytes);
        if (bytes) bulk_g2s(A.ring[i % QRING], P.in + start, bytes, bar);
    };
    if (lane == 0)
        for (uint32_t i = 0; i < QRING; i++) issue(i);
    __syncwarp();

    const bool multi = P.n_seg > 1;
    uint32_t qn = 0;  // queued entries (warp-uniform)
    uint32_t i_fail = 0;
    bool failed = false;
    for (uint32_t i = 0; gw + i * gstride < n_units; i++) {
        const uint32_t u = unit_of(i);
        const uint64_t ustart = (uint64_t)u << SLICE_SHIFT;
        const uint64_t remain = P.n - ustart;
        const uint32_t rem = remain < LIM_MAX ? (uint32_t)remain : LIM_MAX;
        const uint32_t valid = rem < (uint32_t)SLICE ? rem : (uint32_t)SLICE;
        const uint32_t staged = (rem < (uint32_t)QSTAGE ? rem : (uint32_t)QSTAGE) & ~15u;

        // segment ends of this slice: a window of 32 offsets after its start
        uint32_t lima = rem, limb = rem;
        bool general_lims = false;
        if (multi) {
            const uint32_t sf = __ldg(P.unit_seg + u);
            const uint32_t si = sf + lane;
            uint32_t wv = LIM_MAX;
            if (si <= P.n_seg) {
                const uint64_t o = __ldg(P.seg + si);
                const uint64_t r = o > ustart ? o - ustart : 0;
                wv = r < rem ? (uint32_t)r : rem;
            }
            const uint32_t p0 = lane * QBPT;
            uint32_t j = 0;
#pragma unroll
            for (int s = 16; s >= 1; s >>= 1) {
                const uint32_t v = __shfl_sync(0xFFFFFFFFu, wv, j + s - 1);
                if (v <= p0) j += s;
            }
            const uint32_t vj = __shfl_sync(0xFFFFFFFFu, wv, j);
            const uint32_t vj1 = __shfl_sync(0xFFFFFFFFu, wv, j < 31 ? j + 1 : 31);
            const uint32_t last = __shfl_sync(0xFFFFFFFFu, wv, 31);
            if (vj > p0) {
                lima = vj < rem ? vj : rem;
                limb = (j < 31 && vj1 < rem) ? vj1 : rem;
            } else {
                lima = rem;  // beyond the window: handled by the general path
                limb = rem;
            }
            // the window misses boundaries if its last entry is inside the
            // slice, or a lane holds two boundaries within its positions
            const bool need = (last < (uint32_t)SLICE && last < rem) ||
                              (lima < p0 + QBPT && limb < p0 + QBPT);
            general_lims = __any_sync(0xFFFFFFFFu, need);
        }

        const uint32_t s = i % QRING;
        if (!mbar_wait_bounded(&A.bar[s], (i / QRING) & 1)) {
            if (lane == 0) atomicOr(&P.hdr->status, ST_TIMEOUT);
            failed = true;
            i_fail = i;
            break;
        }
        const uint8_t *sb = A.ring[s];
        uint32_t surv, rootm;
        filter_slice<BPS>(P, sb, staged, valid, rem, lima, limb, general_lims, P.seg, ustart, Fs,
                          lane, surv, rootm);
        const uint32_t cnt = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)__popc(surv | rootm));

        if (emit) {
            resolve_slice<W, BPS, VAR>(P, A.q, surv, rootm, sb, u, lima, limb, general_lims,
                                       ustart, rem, Fs, Cs, Es, lane, true);
        } else if (cnt > (uint32_t)QCAP) {
            // too many survivors to queue: count now, emit later
            flush_records<W, VAR>(P, A.q, qn, Fs, Cs, Es, lane);
            qn = 0;
            const uint64_t keys = resolve_slice<W, BPS, VAR>(P, A.q, surv, rootm, sb, u, lima,
                                                             limb, general_lims, ustart, rem, Fs,
                                                             Cs, Es, lane, false);
            if (lane == 0) {
                P.tile_m[u] = UNIT_OVF;
                P.tile_k[u] = keys;
                P.ovf_list[atomicAdd(&P.hdr->ovf_count, 1u)] = u;
            }
        } else {
            if (lane == 0) {
                P.tile_m[u] = 0;  // the slice's last entry sets it when resolved
                P.tile_k[u] = 0;
            }
            __syncwarp();
            if (cnt) {
                if (qn + cnt > (uint32_t)QCAP) {
                    flush_records<W, VAR>(P, A.q, qn, Fs, Cs, Es, lane);
                    qn = 0;
                }
                qn += append_survivors<BPS>(P, A.q, qn, surv, rootm, 0xFFFFFFFFu, sb, u, lima,
                                            limb, general_lims, ustart, rem, lane, 0);
            }
        }
        // the stage is consumed: refill it with the unit QRING ahead
        __syncwarp();
        if (lane == 0) {
            fence_proxy_async_smem();
            issue(i + QRING);
        }
        __syncwarp();
    }
    if (!failed && !emit) flush_records<W, VAR>(P, A.q, qn, Fs, Cs, Es, lane);
    if (failed && lane == 0) {
        // wait (bounded) for this warp's copies that may still be in flight:
        // the stages of units i_fail .. i_fail + QRING - 1
        for (uint32_t i = i_fail; i < i_fail + QRING; i++) {
            if (gw + i * gstride >= n_units) break;
            mbar_wait_bounded(&A.bar[i % QRING], (i / QRING) & 1);
        }
    }
}

}  // namespace pfac

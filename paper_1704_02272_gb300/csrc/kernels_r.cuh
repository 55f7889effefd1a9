// Register-staged scan kernel for 8-bit symbols (alphabets of 129 to 256
// symbols) and 2-bit symbols (alphabets of up to 4, one symbol per byte):
// the walk of Section 2.3 over the compressed records of Section 3.1, with
// the input read from HBM straight into registers.
//
// * Work unit: the 512-byte slice of the queued kernel (same records, key
//   counts and ordering kernels).  A warp takes two consecutive slices per
//   step (pair g = slices 2g and 2g + 1, pairs dealt round-robin over the
//   grid's warps).  Lane l holds bytes 16l .. 16l + 15 of each slice in four
//   registers: one coalesced 16-byte load per lane and slice, issued one step
//   ahead, the pairs further ahead prefetched into L2 by one bulk prefetch.
//   With 2-bit symbols the 16 bytes pack into one word (2 bits a symbol,
//   first symbol lowest).  The symbols after a lane's sixteen (four bytes, or
//   a packed word of sixteen symbols) come from lane l + 1 by a shuffle; for
//   lane 31 of the first slice from lane 0 of the second, for lane 31 of the
//   second from a load of the next pair's head.  Bytes outside the 2-bit
//   range end every window that holds them (those positions walk from the
//   root instead).
// * First stage: each of the lane's 16 positions tests its k-symbol prefix
//   index (or, with the gram filter, its hashed g-symbol string) against a
//   bitmap in shared memory held in 2^REP copies interleaved word by word:
//   lane l reads copy l mod 2^REP, so a warp's 32 random lookups meet fewer
//   bank conflicts.  Per position: one funnel shift forms the index (none at
//   every fourth position), one and-or gives the word address (plus a
//   multiply and a shift for the gram hash), one rotate and one funnel shift
//   move the tested bit into the lane's survivor mask.
// * Second stage, for each candidate (a few per slice), from the registers:
//   the exact prefix bit after the gram filter, the rank of the prefix index
//   (Eq. 1 on the collapsed prefix level) and the child mask of its entry
//   tested with the next symbol; what passes, and positions whose window
//   leaves their segment (walks from the root), join the warp's queue.
// * The queue is resolved in batches through L2 as in the queued kernel (the
//   same resolver and record flush).  A slice with more queue entries than
//   the queue holds is resolved in queue-sized chunks, its record ranks
//   carried from chunk to chunk, so this kernel never needs the counting
//   fallback of the queued kernel; slices with more matched positions than
//   their record space still go to the emit pass.
#pragma once
#include "kernels_q.cuh"

namespace pfac {

constexpr int RNW = 16;       // warps per CTA (default)
constexpr int RNW_WIDE = 24;  // the other choice (80 registers a thread)
constexpr int RPF = 8;        // steps ahead of the L2 prefetch

struct RWarpArea {
    QEntry q[QCAP];
    uint32_t tail[QCAP];   // the resolver's long-walk list (must follow q)
};

__device__ __forceinline__ uint4 ld_stream16(const uint8_t *p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ uint32_t ld_stream4(const uint8_t *p) {
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Predicated forms (no branch): the prefetch or load happens only when on
// is true, and only then is the address used.
__device__ __forceinline__ void prefetch_l2_if(bool on, const void *p, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t"
        "@q cp.async.bulk.prefetch.L2.global [%0], %1;\n\t}" ::"l"(p),
        "r"(bytes), "r"((uint32_t)on)
        : "memory");
}

__device__ __forceinline__ uint32_t ld_stream4_if(bool on, const uint8_t *p) {
    uint32_t v = 0;
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t"
        "@q ld.global.nc.L1::no_allocate.u32 %0, [%1];\n\t}"
        : "+r"(v)
        : "l"(p), "r"((uint32_t)on));
    return v;
}

__device__ __forceinline__ uint4 ld_stream16_if(bool on, const uint8_t *p) {
    uint4 v = make_uint4(0, 0, 0, 0);
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %5, 0;\n\t"
        "@q ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];\n\t}"
        : "+r"(v.x), "+r"(v.y), "+r"(v.z), "+r"(v.w)
        : "l"(p), "r"((uint32_t)on));
    return v;
}

// The lane's symbols as five words: with 8-bit symbols its 16 bytes and the
// 4 bytes after them; with 2-bit symbols its 16 symbols packed in w[0] and
// the next 16 in w[1].

// 16 two-bit symbols (the low bits of 16 bytes) in one word, first symbol
// lowest: per 4-byte word the multiplier places copies at shifts 6, 12, 18
// and 24, so that bits 24 + 2i receive symbol i and no other partial product
// reaches bits 24..31; three byte permutes gather the four top bytes.
__device__ __forceinline__ uint32_t r_pack2(const uint4 &v) {
    const uint32_t b0 = (v.x & 0x03030303u) * 0x01041040u, b1 = (v.y & 0x03030303u) * 0x01041040u;
    const uint32_t b2 = (v.z & 0x03030303u) * 0x01041040u, b3 = (v.w & 0x03030303u) * 0x01041040u;
    return __byte_perm(__byte_perm(b0, b1, 0x0073), __byte_perm(b2, b3, 0x0073), 0x5410);
}

// Bit i set for each byte i of the 16 whose value is 4 or more (outside the
// 2-bit range).
__device__ __forceinline__ uint32_t r_bad2(const uint4 &v) {
    const uint32_t x[4] = {v.x, v.y, v.z, v.w};
    uint32_t m = 0;
#pragma unroll
    for (int w = 0; w < 4; w++)
#pragma unroll
        for (int b = 0; b < 4; b++)
            if ((x[w] >> (8 * b)) & 0xFCu) m |= 1u << (4 * w + b);
    return m;
}

// Symbols j .. of the lane's window for a compile-time j < 16 (the low bits
// of the result: four bytes, or sixteen 2-bit symbols).
template <int BPS>
__device__ __forceinline__ uint32_t r_twin(const uint32_t (&w)[5], int j) {
    if (BPS == 2) return j == 0 ? w[0] : __funnelshift_r(w[0], w[1], 2 * j);
    return (j & 3) ? __funnelshift_r(w[j >> 2], w[(j >> 2) + 1], 8 * (j & 3)) : w[j >> 2];
}

// The same for a run-time j (8-bit symbols: a select chain instead of an
// indexed register access).
template <int BPS>
__device__ __forceinline__ uint32_t r_window(const uint32_t (&w)[5], uint32_t j) {
    if (BPS == 2) return __funnelshift_r(w[0], w[1], 2 * j);
    const uint32_t i = j >> 2;
    uint32_t lo = w[0], hi = w[1];
    if (i == 1) { lo = w[1]; hi = w[2]; }
    if (i == 2) { lo = w[2]; hi = w[3]; }
    if (i == 3) { lo = w[3]; hi = w[4]; }
    return __funnelshift_r(lo, hi, 8 * (j & 3));
}

// Word address of position window t in the first-stage table: for the
// prefix bitmap the index's bits above the bit number (t >> 5) placed at bit
// REP + 2; for the gram filter the top bits of the hash t * gm (table.h),
// taken by a high multiply by gmh = 2^(word bits + REP + 2) so that the
// shift runs on the multiply pipe.  amask keeps the word bits, c4 selects
// the lane's copy.
template <int REP, int GRAM>
__device__ __forceinline__ uint32_t r_addr(uint32_t t, uint32_t c4, uint32_t amask, uint32_t gm,
                                           uint32_t gmh) {
    if (GRAM) return (__umulhi(t * gm, gmh) & amask) | c4;
    return ((REP >= 3 ? (t << (REP - 3)) : (t >> (3 - REP))) & amask) | c4;
}

// First stage of one slice for the lane's 16 positions (bit j of the result
// set when position j's window passes the filter): fewer registers than the
// two-slice form, for the wider CTA.
template <int BPS, int REP, int GRAM>
__device__ __forceinline__ uint32_t r_first_stage1(const MatchParams &P, const uint32_t (&w)[5],
                                                   uint32_t c4, uint32_t amask, uint32_t gm,
                                                   uint32_t gmh, uint32_t tbytes) {
    extern __shared__ __align__(128) uint8_t smem[];
    uint32_t acc[2] = {0, 0};
#pragma unroll
    for (int j = 0; j < 16; j++) {
        const uint32_t t = r_twin<BPS>(w, j);
        const uint32_t x = *reinterpret_cast<const uint32_t *>(
            smem + chk(P, r_addr<REP, GRAM>(t, c4, amask, gm, gmh), tbytes));
        acc[j >> 3] = __funnelshift_r(acc[j >> 3], __funnelshift_r(x, x, t), 1);
    }
    return (acc[0] >> 24) | ((acc[1] >> 16) & 0xFF00u);
}

// First stage of the two slices of a step for the lane's 16 positions in
// each (their 32 lookups independent, so they overlap): bit j of sa / sb is
// set when position j's window passes the filter.  The first-stage table
// sits at the start of the dynamic shared memory, so a lookup needs no base
// register.  Each slice's bits gather in two chains of eight.
template <int BPS, int REP, int GRAM>
__device__ __forceinline__ void r_first_stage2(const MatchParams &P, const uint32_t (&wa)[5],
                                               const uint32_t (&wb)[5], uint32_t c4,
                                               uint32_t amask, uint32_t gm, uint32_t gmh,
                                               uint32_t tbytes, uint32_t &sa, uint32_t &sb) {
    extern __shared__ __align__(128) uint8_t smem[];
    uint32_t acc_a[2] = {0, 0}, acc_b[2] = {0, 0};
#pragma unroll
    for (int j = 0; j < 16; j++) {
        const uint32_t ta = r_twin<BPS>(wa, j), tb = r_twin<BPS>(wb, j);
        const uint32_t xa = *reinterpret_cast<const uint32_t *>(
            smem + chk(P, r_addr<REP, GRAM>(ta, c4, amask, gm, gmh), tbytes));
        const uint32_t xb = *reinterpret_cast<const uint32_t *>(
            smem + chk(P, r_addr<REP, GRAM>(tb, c4, amask, gm, gmh), tbytes));
        // bit t & 31 of each word to bit 0, then into the top of acc
        acc_a[j >> 3] = __funnelshift_r(acc_a[j >> 3], __funnelshift_r(xa, xa, ta), 1);
        acc_b[j >> 3] = __funnelshift_r(acc_b[j >> 3], __funnelshift_r(xb, xb, tb), 1);
    }
    // positions 0..7 end at bits 24..31 of the first chain, 8..15 of the second
    sa = (acc_a[0] >> 24) | ((acc_a[1] >> 16) & 0xFF00u);
    sb = (acc_b[0] >> 24) | ((acc_b[1] >> 16) & 0xFF00u);
}

// Second stage of one candidate whose window (symbols j ..) is t: prefix
// index x = the first k symbols.  With the gram filter the exact bit
// of x in F_k must be set.  With child masks, and when the next symbol lies
// inside the walk's limit, the entry's mask must hold that symbol's bit (an
// entry that reports output has an all-ones mask); a symbol outside the
// alphabet ends every other walk.
template <int BPS, int GRAM>
__device__ __forceinline__ bool r_keep(const MatchParams &P, uint32_t t, bool has_next,
                                       const uint32_t *Fs, const uint32_t *Cs, const uint32_t *Ms,
                                       uint32_t &x) {
    const uint32_t kb = BPS * P.k;
    x = kb >= 32 ? t : (t & ((1u << kb) - 1u));
    x = (uint32_t)chk(P, x, 1ull << kb);
    if (GRAM) {
        const uint32_t fw = Fs[(x >> 5) << P.rep_log2];
        if (!((fw >> (x & 31)) & 1u)) return false;
    }
    if (!P.tbl_m_words || !has_next) return true;
    const uint32_t r = (uint32_t)chk(P, prefix_rank(Fs, P.rep_log2, Cs, P.c_shift, x), P.T.n_e[P.k]);
    const uint32_t sigma = P.T.sigma;
    const uint32_t mb = mask_bits(sigma), ones = mb == 32 ? 0xFFFFFFFFu : (1u << mb) - 1u;
    const uint32_t mi = (uint32_t)chk(P, mb == 32 ? r : (r * mb) >> 5, P.tbl_m_words);
    const uint32_t mr = mb == 32 ? Ms[mi] : (Ms[mi] >> ((r * mb) & 31)) & ones;
    const uint32_t c = (t >> kb) & ((1u << BPS) - 1u);
    return c < sigma ? ((mr >> child_hash(c, sigma)) & 1u) != 0 : mr == ones;
}

// Positions of one lane's 16 whose k-symbol window lies inside their segment
// and the staged bytes (fv), and positions inside their segment at all (ex),
// for slices where a segment ends or the input stops; as in the queued
// kernel's filter.
__device__ __forceinline__ void r_window_masks(const MatchParams &P, uint32_t p0, uint32_t kf,
                                               uint32_t valid, uint32_t staged, uint32_t rem,
                                               uint32_t lima, uint32_t limb, bool general,
                                               uint64_t ustart, uint32_t &fv, uint32_t &ex) {
    fv = 0;
    ex = 0;
    if (p0 >= valid) return;
    if (!general) {
        auto below = [&](uint32_t x) -> uint32_t {  // positions p0 + j < x
            const uint32_t n = x > p0 ? (x - p0 < 16u ? x - p0 : 16u) : 0u;
            return n >= 32 ? 0xFFFFFFFFu : (1u << n) - 1u;
        };
        const uint32_t in_a = below(lima), vm = below(valid);
        const uint32_t la = lima < staged ? lima : staged, lb = limb < staged ? limb : staged;
        const uint32_t fa = la >= kf ? below(la - kf + 1) : 0u;  // p + kf <= la
        const uint32_t fb = lb >= kf ? below(lb - kf + 1) : 0u;
        ex = (in_a | below(limb)) & vm;
        fv = ((fa & in_a) | (fb & ~in_a)) & vm;
        return;
    }
#pragma unroll 1
    for (uint32_t j = 0; j < 16; j++) {
        const uint32_t p = p0 + j;
        if (p >= valid) break;
        const uint32_t lj = lim_of(P, p, lima, limb, true, ustart, rem);
        if (lj > p) ex |= 1u << j;
        const uint32_t lw = lj < staged ? lj : staged;
        if (p + kf <= lw) fv |= 1u << j;
    }
}

// Segment ends of one slice for its lanes (multi-segment inputs): lima = the
// first offset above the lane's first position, limb = the one after;
// general = some lane's positions meet more than that (or the window of 32
// offsets ends inside the slice), the exact limit then found by search.
__device__ __forceinline__ void r_seg_limits(const MatchParams &P, uint32_t u, uint64_t ustart,
                                             uint32_t rem, uint32_t lane, uint32_t &lima,
                                             uint32_t &limb, bool &general) {
    const uint32_t sf = __ldg(P.unit_seg + u);
    const uint32_t si = sf + lane;
    const uint64_t o = si <= P.n_seg ? __ldg(P.seg + si) : ~0ull;
    uint32_t wv = LIM_MAX;
    if (o != ~0ull) {
        const uint64_t r = o > ustart ? o - ustart : 0;
        wv = r < rem ? (uint32_t)r : rem;
    }
    const uint32_t w0 = __shfl_sync(0xFFFFFFFFu, wv, 0);
    const uint32_t w1 = __shfl_sync(0xFFFFFFFFu, wv, 1);
    general = false;
    if (w0 >= (uint32_t)(SLICE + 16)) {
        // no segment end inside the slice or its halo: one limit for every lane
        lima = w0 < rem ? w0 : rem;
        limb = w1 < rem ? w1 : rem;
        return;
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
        lima = rem;
        limb = rem;
    }
    const bool need = (last < (uint32_t)SLICE && last < rem) || (lima < p0 + QBPT && limb < p0 + QBPT);
    general = __any_sync(0xFFFFFFFFu, need);
}

struct RQueue {
    uint32_t qn;          // entries queued (warp-uniform)
    uint32_t carry_unit;  // slice continued into the next batch (UNIT_OVF: none)
    uint32_t carry;       // its records in earlier batches
};

// Resolves the warp's queue out of line: a rare path (once per queue of
// survivors), kept out of the streaming loop so that the loop's code and
// registers stay small.  P points at the kernel's parameter block.
template <int W, int VAR>
__device__ __noinline__ uint2 r_flush(const MatchParams *P, QEntry *q, uint32_t n,
                                      const uint32_t *Fs, const uint32_t *Cs, const uint32_t *Es,
                                      uint32_t lane, uint32_t carry_unit, uint32_t carry) {
    flush_records_c<W, VAR>(*P, q, n, Fs, Cs, Es, lane, carry_unit, carry);
    return make_uint2(carry_unit, carry);
}

// Empties the warp's queue: a queue of whole slices (whole = its last entry
// ends a slice, and no slice continues from an earlier batch) goes to the
// resolver kernel while its buffers have room; otherwise the warp resolves
// it now.
template <int W, int VAR>
__device__ __forceinline__ void r_flush_queue(const MatchParams &P, RWarpArea &A, RQueue &Q,
                                              const uint32_t *Fs, const uint32_t *Cs,
                                              const uint32_t *Es, uint32_t lane,
                                              bool whole = true) {
    if (whole && Q.carry_unit == UNIT_OVF && defer_queue(P, A.q, Q.qn, lane)) {
        Q.qn = 0;
        return;
    }
    const uint2 c = r_flush<W, VAR>(&P, A.q, Q.qn, Fs, Cs, Es, lane, Q.carry_unit, Q.carry);
    Q.carry_unit = c.x;
    Q.carry = c.y;
    Q.qn = 0;
}

// Appends the lane's queue entries (the bits of keep | root, in position
// order; the lanes in lane order) for slice `unit`; resolves the queue first
// when they do not fit, and resolves in queue-sized chunks a slice that alone
// has more entries than the queue holds.
template <int BPS, int W, int VAR>
__device__ __forceinline__ void r_append(const MatchParams &P, RWarpArea &A, RQueue &Q,
                                         uint32_t keep, uint32_t root, const uint32_t (&w)[5],
                                         uint32_t unit, uint32_t lima, uint32_t limb,
                                         bool general, uint64_t ustart, uint32_t rem,
                                         const uint32_t *Fs, const uint32_t *Cs,
                                         const uint32_t *Es, uint32_t lane) {
    const uint32_t m = keep | root;
    const uint32_t c = __popc(m);
    uint32_t inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t nb = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= (uint32_t)o) inc += nb;
    }
    const uint32_t tot = __shfl_sync(0xFFFFFFFFu, inc, 31);
    if (tot == 0) return;
    const uint32_t excl = inc - c;
    if (Q.qn + tot > (uint32_t)QCAP && Q.qn) r_flush_queue<W, VAR>(P, A, Q, Fs, Cs, Es, lane);
    const uint32_t p0 = lane * QBPT;
    const uint32_t kb = BPS * P.k, kmask = kb >= 32 ? 0xFFFFFFFFu : (1u << kb) - 1u;
    // walks stop at the input end (a clean slice's limits do not say where)
    const uint64_t remain = P.n - ustart;
    const uint32_t rem_x = remain < LIM_MAX ? (uint32_t)remain : LIM_MAX;
    for (uint32_t done = 0;;) {
        const uint32_t room = QCAP - Q.qn;
        const uint32_t take = tot - done < room ? tot - done : room;
        uint32_t mm = m, e = excl;
        while (mm) {
            const uint32_t j = __ffs(mm) - 1;
            mm &= mm - 1;
            if (e >= done && e < done + take) {
                const uint32_t p = p0 + j, slot = e - done;
                QEntry en;
                en.unit = unit;
                en.pos = p | (slot << 10) | (e + 1 == tot ? LAST_FLAG : 0u);
                en.x = ((root >> j) & 1u) ? ROOT_X : (r_window<BPS>(w, j) & kmask);
                const uint32_t lj = lim_of(P, p, lima, limb, general, ustart, rem);
                en.lim = lj < rem_x ? lj : rem_x;
                A.q[chk(P, Q.qn + slot, QCAP)] = en;
            }
            e++;
        }
        __syncwarp();
        Q.qn += take;
        done += take;
        if (done == tot) break;
        // the queue is full and the slice goes on: resolve, carrying its ranks
        r_flush_queue<W, VAR>(P, A, Q, Fs, Cs, Es, lane, false);
    }
}

// One slice after its first stage (surv): window masks, second stage, queue.
template <int BPS, int W, int GRAM, int VAR>
__device__ __forceinline__ void r_slice(const MatchParams &P, RWarpArea &A, RQueue &Q,
                                        const uint32_t (&w)[5], uint32_t surv, bool halo_ok,
                                        uint32_t u, bool clean, uint32_t bad, const uint32_t *Fs,
                                        const uint32_t *Cs, const uint32_t *Es,
                                        const uint32_t *Ms, uint32_t lane) {
    // symbols held past the slice: 4 bytes, or 16 packed 2-bit symbols
    constexpr uint32_t HALO = BPS == 8 ? 4u : 16u;
    const uint64_t ustart = (uint64_t)u << SLICE_SHIFT;
    const uint32_t p0 = lane * QBPT;
    // a clean slice (one segment; the slice, its 4-byte halo and every
    // start inside the input and below starts_end) needs no limits: every
    // position starts a walk and every window is held in registers; the
    // exact input end is applied when survivors are queued
    uint32_t rem = LIM_MAX, valid = SLICE, staged = SLICE + HALO, lima = LIM_MAX, limb = LIM_MAX;
    bool general = false;
    uint32_t fv = 0xFFFFu, ex = 0xFFFFu;
    if (!clean) {
        const uint64_t remain = P.n - ustart;
        rem = remain < LIM_MAX ? (uint32_t)remain : LIM_MAX;
        valid = rem < (uint32_t)SLICE ? rem : (uint32_t)SLICE;
        const uint64_t sl = P.starts_end > ustart ? P.starts_end - ustart : 0;
        if (sl < valid) valid = (uint32_t)sl;
        // bytes held in registers: whole 16-byte chunks, then (halo_ok) the
        // 4-byte head of the next slice
        staged = rem < (uint32_t)SLICE ? rem & ~15u : (uint32_t)SLICE + (halo_ok ? HALO : 0u);
        lima = limb = rem;
        if (P.n_seg > 1) r_seg_limits(P, u, ustart, rem, lane, lima, limb, general);
        const uint32_t kf = P.kf;
        const uint32_t lim0 = lima < staged ? lima : staged;
        if (general || p0 + QBPT - 1 + kf > lim0 || p0 + QBPT > valid)
            r_window_masks(P, p0, kf, valid, staged, rem, lima, limb, general, ustart, fv, ex);
    }
    if (BPS < 8 && __any_sync(0xFFFFFFFFu, bad != 0)) {
        // windows holding a byte outside the packed symbol range (bit i of
        // bad: symbol i of the lane's 32, its 16 and the next 16)
        const uint32_t kf = P.kf;
        uint32_t bw = 0;
        for (uint32_t t = 0; t < kf; t++) bw |= bad >> t;
        fv &= ~bw;
    }
    surv &= fv;
    const uint32_t root = ex & ~fv;
    // second stage over the lane's candidates
    uint32_t keep = 0;
    const uint32_t k = P.k;
    uint32_t mm = surv;
    while (mm) {
        const uint32_t j = __ffs(mm) - 1;
        mm &= mm - 1;
        const uint32_t p = p0 + j;
        const uint32_t t = r_window<BPS>(w, j);
        // the next symbol is held in registers and inside the walk's limit
        const bool has_next =
            p + k < staged && p + k < lim_of(P, p, lima, limb, general, ustart, rem);
        uint32_t x;
        if (r_keep<BPS, GRAM>(P, t, has_next, Fs, Cs, Ms, x)) keep |= 1u << j;
    }
    if (__any_sync(0xFFFFFFFFu, (keep | root) != 0))
        r_append<BPS, W, VAR>(P, A, Q, keep, root, w, u, lima, limb, general, ustart, rem, Fs, Cs,
                              Es, lane);
}

// The scan pass of the compressed layout with 8-bit symbols.  The int
// argument is unused (the launch signature is shared with the other scan
// kernels).
template <int BPS, int W, int REP, int GRAM, int VAR, int NW>
__global__ void __launch_bounds__(NW * 32, 1) k_scanr(const __grid_constant__ MatchParams P,
                                                      const int) {
    constexpr uint32_t RTHREADS = NW * 32;
    constexpr uint32_t HALO = BPS == 8 ? 4u : 16u;  // bytes of the next pair's head a step holds
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t n_units = P.n_tiles;
    const uint32_t n_pairs = (n_units + 1) >> 1;
    const uint32_t gw = blockIdx.x * NW + warp, gstride = gridDim.x * NW;
    if (blockIdx.x * NW >= n_pairs) return;  // the whole CTA has no pair

    // the first-stage table at offset 0: the gram filter, or the prefix
    // bitmap copies when there is none
    uint32_t *Gs = reinterpret_cast<uint32_t *>(smem);
    uint32_t *Fs = Gs + P.tbl_g_words;
    uint32_t *Cs = Fs + P.tbl_words;
    uint32_t *Es = Cs + P.tbl_c_words;
    uint32_t *Ms = Es + P.tbl_e_words;
    RWarpArea *areas = reinterpret_cast<RWarpArea *>(
        smem + ((((size_t)P.tbl_words + P.tbl_c_words + P.tbl_e_words + P.tbl_m_words +
                  P.tbl_g_words) * 4 + 127) & ~(size_t)127));
    {
        const uint32_t rep = P.rep_log2;
        for (uint32_t i = threadIdx.x; i < P.tbl_words; i += RTHREADS) Fs[i] = __ldg(P.F + (i >> rep));
        for (uint32_t i = threadIdx.x; i < P.tbl_c_words; i += RTHREADS) Cs[i] = __ldg(P.C + i);
        if (VAR == VAR_FE)
            for (uint32_t i = threadIdx.x; i < P.tbl_e_words; i += RTHREADS) Es[i] = __ldg(P.E + i);
        for (uint32_t i = threadIdx.x; i < P.tbl_m_words; i += RTHREADS) Ms[i] = __ldg(P.M + i);
        // gram filter: word w of each copy is the OR of 2^g_fold table words
        const uint32_t gr = P.g_rep, gf = P.g_fold;
        for (uint32_t i = threadIdx.x; i < P.tbl_g_words; i += RTHREADS) {
            const uint32_t *src = P.T.G + ((size_t)(i >> gr) << gf);
            uint32_t v = 0;
            for (uint32_t f = 0; f < (1u << gf); f++) v |= __ldg(src + f);
            Gs[i] = v;
        }
    }
    __syncthreads();
    RWarpArea &A = areas[warp];

    // first-stage constants: the lane's copy, the address mask, the hash,
    // the table's bytes
    const uint32_t c4 = (lane & ((1u << REP) - 1u)) << 2;
    const uint32_t tbytes = (GRAM ? P.tbl_g_words : P.tbl_words) * 4u;
    uint32_t amask, gm = 0, gmh = 0;
    if (GRAM) {
        const uint32_t hbw = P.g_hb - 5;
        gm = gram_mul(BPS * P.kf);
        gmh = 1u << (hbw + REP + 2);  // high word of y * gmh: the word at bit REP + 2
        amask = ((1u << hbw) - 1u) << (REP + 2);
    } else {
        amask = ((1u << (BPS * P.k - 5u)) - 1u) << (REP + 2);
    }

    const uint64_t N = P.n;
    // clean pairs (every load in bounds, the next pair's head too, every
    // start below starts_end, one segment) take loads without checks and
    // slices without limits: pairs g < g_clean
    uint32_t g_clean = 0;
    if (P.n_seg <= 1 && N >= HALO) {
        const uint64_t a = (N - HALO) >> (SLICE_SHIFT + 1), b = P.starts_end >> (SLICE_SHIFT + 1);
        const uint64_t c = a < b ? a : b;
        g_clean = c < n_pairs ? (uint32_t)c : n_pairs;
    }
    const uint32_t it_clean = gw < g_clean ? (g_clean - gw + gstride - 1) / gstride : 0u;
    const uint64_t step_b = (uint64_t)gstride << (SLICE_SHIFT + 1);
    const uint8_t *lane_ptr = P.in + ((uint64_t)gw << (SLICE_SHIFT + 1)) + lane * 16u;
    const bool l31 = lane == 31, l0 = lane == 0;
    // lane 31 also loads the next pair's head: 4 bytes, or 16 with 2-bit
    // symbols (h.y .. h.w stay zero with 8-bit symbols)
    auto load_head = [&](bool on, const uint8_t *q) -> uint4 {
        if (BPS == 8) return make_uint4(ld_stream4_if(on, q), 0u, 0u, 0u);
        return ld_stream16_if(on, q);
    };
    auto load_pair = [&](uint32_t i, uint4 &a, uint4 &b, uint4 &h) {
        const uint8_t *q = lane_ptr + i * step_b;
        if (i < it_clean) {
            a = ld_stream16(q);
            b = ld_stream16(q + SLICE);
            h = load_head(l31, q + SLICE + 16);
            return;
        }
        a = make_uint4(0, 0, 0, 0);
        b = a;
        h = a;
        const uint32_t g = gw + i * gstride;
        if (g >= n_pairs) return;
        const uint64_t s0 = (uint64_t)g << (SLICE_SHIFT + 1);
        const uint64_t o0 = s0 + lane * 16u, o1 = o0 + SLICE;
        if (o0 + 16 <= N) a = ld_stream16(P.in + o0);
        if (o1 + 16 <= N) b = ld_stream16(P.in + o1);
        h = load_head(l31 && s0 + 2 * SLICE + HALO <= N, P.in + s0 + 2 * SLICE);
    };
    // the L2 prefetch runs RPF steps ahead over the clean pairs
    const uint8_t *pair_ptr = P.in + ((uint64_t)gw << (SLICE_SHIFT + 1));
    for (uint32_t i = 0; i < RPF && i < it_clean; i++)
        prefetch_l2_if(l0, pair_ptr + i * step_b, 2 * SLICE);

    RQueue Q{0u, UNIT_OVF, 0u};
    // one step: pair i, its registers loaded the step before
    auto step = [&](uint32_t i, const uint4 &ca, const uint4 &cb, const uint4 &ch) {
        prefetch_l2_if(l0 && i + RPF < it_clean, pair_ptr + (i + RPF) * step_b, 2 * SLICE);
        const uint32_t g = gw + i * gstride;
        const bool clean = i < it_clean;
        // each lane's symbols: its own and the following ones, from the next
        // lane; lane 31 takes the second slice's lane 0 (first slice) or the
        // next pair's head (second slice)
        uint32_t wa[5], wb[5], bad_a = 0, bad_b = 0;
        if (BPS == 8) {
            const uint32_t a_next = __shfl_down_sync(0xFFFFFFFFu, ca.x, 1);
            const uint32_t b_next = __shfl_down_sync(0xFFFFFFFFu, cb.x, 1);
            const uint32_t b_first = __shfl_sync(0xFFFFFFFFu, cb.x, 0);
            wa[0] = ca.x; wa[1] = ca.y; wa[2] = ca.z; wa[3] = ca.w;
            wa[4] = l31 ? b_first : a_next;
            wb[0] = cb.x; wb[1] = cb.y; wb[2] = cb.z; wb[3] = cb.w;
            wb[4] = l31 ? ch.x : b_next;
        } else {
            const uint32_t pa = r_pack2(ca), pb = r_pack2(cb), ph = r_pack2(ch);
            const uint32_t a_next = __shfl_down_sync(0xFFFFFFFFu, pa, 1);
            const uint32_t b_next = __shfl_down_sync(0xFFFFFFFFu, pb, 1);
            const uint32_t b_first = __shfl_sync(0xFFFFFFFFu, pb, 0);
            wa[0] = pa;
            wa[1] = l31 ? b_first : a_next;
            wb[0] = pb;
            wb[1] = l31 ? ph : b_next;
            wa[2] = wa[3] = wa[4] = wb[2] = wb[3] = wb[4] = 0;
            // bytes outside the 2-bit range, rare: their masks only then
            const uint32_t hi = 0xFCFCFCFCu;
            const uint32_t any = ((ca.x | ca.y | ca.z | ca.w | cb.x | cb.y | cb.z | cb.w) & hi) |
                                 ((ch.x | ch.y | ch.z | ch.w) & hi);
            if (__any_sync(0xFFFFFFFFu, any != 0)) {
                const uint32_t ma = r_bad2(ca), mb = r_bad2(cb), mh = r_bad2(ch);
                const uint32_t ma_next = __shfl_down_sync(0xFFFFFFFFu, ma, 1);
                const uint32_t mb_next = __shfl_down_sync(0xFFFFFFFFu, mb, 1);
                const uint32_t mb_first = __shfl_sync(0xFFFFFFFFu, mb, 0);
                bad_a = ma | ((l31 ? mb_first : ma_next) << 16);
                bad_b = mb | ((l31 ? mh : mb_next) << 16);
            }
        }
        uint32_t sa, sb;
        if (NW == RNW) {
            r_first_stage2<BPS, REP, GRAM>(P, wa, wb, c4, amask, gm, gmh, tbytes, sa, sb);
        } else {
            sa = r_first_stage1<BPS, REP, GRAM>(P, wa, c4, amask, gm, gmh, tbytes);
            sb = r_first_stage1<BPS, REP, GRAM>(P, wb, c4, amask, gm, gmh, tbytes);
        }
        // the head of slice 2g + 1 is held when its lane 0 chunk was loaded,
        // that of the next pair when lane 31 loaded it
        const uint64_t s1 = ((uint64_t)2 * g + 1) << SLICE_SHIFT;
        r_slice<BPS, W, GRAM, VAR>(P, A, Q, wa, sa, clean || s1 + 16 <= N, 2 * g, clean, bad_a, Fs,
                                   Cs, Es, Ms, lane);
        if (clean || 2 * g + 1 < n_units)
            r_slice<BPS, W, GRAM, VAR>(P, A, Q, wb, sb, clean || s1 + SLICE + HALO <= N, 2 * g + 1,
                                       clean, bad_b, Fs, Cs, Es, Ms, lane);
    };
    // this step's registers and the next step's, loaded a step ahead
    uint4 a0, b0, a1, b1;
    uint4 h0, h1;
    load_pair(0, a0, b0, h0);
    for (uint32_t i = 0; gw + i * gstride < n_pairs; i++) {
        load_pair(i + 1, a1, b1, h1);
        step(i, a0, b0, h0);
        a0 = a1;
        b0 = b1;
        h0 = h1;
    }
    if (Q.qn) r_flush_queue<W, VAR>(P, A, Q, Fs, Cs, Es, lane);
}


// The resolver kernel: each warp takes batches the scan kernel handed over (whole slices, in queue order), resolves them with
// the prefix node's bitmap, counts and entries read through L2 (P has one
// bitmap copy), and writes their records and counts as the scan kernel would
// have.
// The batches are chains of dependent L2 loads: occupancy (RES_CTAS CTAs of
// RES_WARPS warps on every SM, at most 64 registers a thread) is what
// hides them.
constexpr int RES_WARPS = 8;
constexpr int RES_CTAS = 4;

template <int W>
__global__ void __launch_bounds__(RES_WARPS * 32, RES_CTAS)
    k_resolve(const __grid_constant__ MatchParams P) {
    __shared__ RWarpArea areas[RES_WARPS];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    RWarpArea &A = areas[warp];
    const uint32_t nb0 = *(volatile uint32_t *)&P.hdr->defer_batches;
    const uint32_t nb = nb0 < P.dbatch_cap ? nb0 : P.dbatch_cap;
    const uint32_t gw = blockIdx.x * RES_WARPS + warp, gs = gridDim.x * RES_WARPS;
    for (uint32_t b = gw; b < nb; b += gs) {
        const uint2 d = P.dbatch[b];
        if (d.y == 0 || d.y > (uint32_t)QCAP) continue;
        for (uint32_t i = lane; i < d.y; i += 32)
            *reinterpret_cast<uint4 *>(&A.q[i]) = P.defer[chk(P, (uint64_t)d.x + i, P.defer_cap)];
        __syncwarp();
        uint32_t cu = UNIT_OVF, cc = 0;
        flush_records_c<W, VAR_F | VAR_RES>(P, A.q, d.y, P.F, P.C, nullptr, lane, cu, cc);
        __syncwarp();
    }
}

}  // namespace pfac

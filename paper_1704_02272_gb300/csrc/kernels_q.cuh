// Queued scan kernel for the compressed layout (Section 2.3 walk over the
// Section 3.1 records), built so that no warp waits for another.
//
// * Work unit: a 512-byte slice of the input.  Slice g goes to global warp
//   g mod (warps in the grid); every warp streams its own slices with
//   cp.async.bulk into a private 4-stage ring of 528-byte stages (slice plus
//   a 16-byte halo), each stage with its own mbarrier.  CTAs have 16 or 24
//   warps.
// * First stage: each lane owns 16 start positions of the slice and tests
//   each against a table in shared memory: the depth-k prefix bitmap F_k
//   (replicated over bank groups so a warp's 32 random lookups conflict
//   little), the prefix bytes B_k (one byte per index), or the hashed gram
//   filter G over the next g symbols.  Positions whose window is not
//   available (segment end, input end, symbol outside the packed range)
//   become "root" survivors that walk from the root.
// * Second stage, per candidate: the exact F_k bit (after G), the bucket of
//   the next symbol (after B_k), the child mask of the entry (M_k).
// * Survivors go to a per-warp queue in shared memory.  When a slice's do
//   not fit, the warp resolves the queue in one batch: four queue entries
//   per lane, all advanced in lockstep, so each lane keeps several
//   independent loads in flight.  Resolution ranks the prefix index in F_k
//   (block counts C_k plus popcounts, Eq. 1 applied to the prefix level) to
//   read its entry E_k (the state at depth k or the output of a walk that
//   stopped earlier), walks the records through L2 one level per round, and
//   finishes long walks one per lane along consecutive chain records.
// * Output: per slice, the survivors' (position, fin) records in position
//   order plus the slice's key count; slices with more matches than their
//   record space are resolved immediately in quarters (counting only) and
//   re-run by the emit pass, which writes their keys directly.
#pragma once
#include "kernels.cuh"

namespace pfac {

constexpr int QW = 16;                   // warps per CTA (default; 24 is the other choice)
constexpr int QW_WIDE = 24;
constexpr int QBPT = 16;                 // start positions per lane per slice
constexpr int SLICE = 32 * QBPT;         // 512 start positions per slice
constexpr int SLICE_SHIFT = 9;
constexpr int QRING = 4;                 // stages per warp ring
constexpr int QSTAGE = SLICE + 16;       // bytes per stage: slice plus halo
constexpr int SCAP = 32;                 // match records kept per slice by the scan pass
constexpr int QCAP = 128;                // queue entries per warp (and most survivors
                                         // of one slice queued at once)
constexpr int QU = QCAP / 32;            // queue entries per lane per batch
// walks a lane advances together while resolving: fewer for 48-byte records
__host__ __device__ constexpr int walks_per_lane(int W) { return W == 8 ? 2 : 4; }
// walks per lane of one resolve pass: fewer in the resolver kernel
__host__ __device__ constexpr int pass_walks(int W, int VAR) {
    return (VAR & VAR_RES) ? (W == 8 ? 1 : 2) : walks_per_lane(W);
}
constexpr uint32_t ROOT_X = 0xFFFFFFFFu; // queue entry: walk from the root
constexpr uint32_t DAG_PENDING = 0x80000000u;  // resolved entry: merged-trie walk still to run
constexpr uint32_t LAST_FLAG = 0x80000000u;  // queue entry: the slice's last
constexpr uint32_t UNIT_OVF = 0xFFFFFFFFu;
constexpr uint32_t LIM_MAX = 0xFFFFFFF0u;

struct QEntry {
    uint32_t unit;
    uint32_t pos;   // position in the slice | slot << 10 | LAST_FLAG on the slice's last
    uint32_t x;     // prefix index, or ROOT_X
    uint32_t lim;   // walk limit relative to the slice start
};

struct WarpArea {
    uint8_t ring[QRING][QSTAGE];
    QEntry q[QCAP];
    uint32_t tail[QCAP];      // long walks compacted during resolution
    uint64_t bar[QRING];
};

// Rank of prefix index x among the set bits of F_k (Eq. 1 on the prefix
// level): the count before its word (or 8-word group) plus popcounts.
__device__ __forceinline__ uint32_t prefix_rank(const uint32_t *Fs, uint32_t rep,
                                                const uint32_t *Cs, uint32_t cshift, uint32_t x) {
    const uint32_t w = x >> 5;
    uint32_t r = Cs[w >> cshift] + __popc(Fs[w << rep] & ((1u << (x & 31)) - 1u));
    if (cshift) {
        const uint32_t b0 = (w >> 3) << 3;
        if (rep == 0) {
            // one 8-word group, two vector loads, words before w only
            const uint4 g0 = *reinterpret_cast<const uint4 *>(Fs + b0);
            const uint4 g1 = *reinterpret_cast<const uint4 *>(Fs + b0 + 4);
            const uint32_t o = w & 7;
            r += (o > 0 ? __popc(g0.x) : 0) + (o > 1 ? __popc(g0.y) : 0) +
                 (o > 2 ? __popc(g0.z) : 0) + (o > 3 ? __popc(g0.w) : 0) +
                 (o > 4 ? __popc(g1.x) : 0) + (o > 5 ? __popc(g1.y) : 0) +
                 (o > 6 ? __popc(g1.z) : 0);
        } else {
            for (uint32_t i = b0; i < w; i++) r += __popc(Fs[i << rep]);
        }
    }
    return r;
}

// Record words of state r needed to take a step on symbol c: the word
// holding c's bit, the rank base below that word, the meta word and (for
// sigma > 32) the state's output.  A packed record (W == 0) is its own meta
// word: the all-leaf flag at bit 31 and the base below bit aux, the bitmap
// between.  A row of the dense transition table (W == 3, aux = sigma) gives
// the child itself: the step then sees a one-bit bitmap and the child as its
// base.
template <int W>
__device__ __forceinline__ void load_step(const uint32_t *__restrict__ rec, uint32_t r, uint32_t c,
                                          uint32_t &word, uint32_t &below, uint32_t &meta,
                                          uint32_t &f, uint32_t aux = 0) {
    constexpr int RW = rec_words(W);
    const uint32_t *R = rec + (size_t)r * RW;
    const uint32_t psh = aux;
    if (W == 3) {
        const uint32_t nx = c < aux ? __ldg(rec + (size_t)r * aux + c) : 0u;
        word = nx ? 1u << (c & 31) : 0u;
        below = 0;
        meta = nx;
        f = 0;
    } else if (W == 0) {
        const uint32_t v = __ldg(R);
        word = v >> psh;  // the flag lands above the bitmap, past every symbol
        below = 0;
        meta = v;
        f = 0;
    } else if (W == 1) {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(R));
        word = v.x;
        below = 0;
        meta = v.y;
        f = 0;
    } else if (W == 2) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(R));
        word = (c & 32) ? v.y : v.x;
        below = (c & 32) ? (uint32_t)__popc(v.x) : 0u;
        meta = v.z;
        f = v.w;
    } else {
        const uint32_t wi = (c >> 5) & 7;
        word = __ldg(R + wi);
        const uint2 mf = __ldg(reinterpret_cast<const uint2 *>(R + 8));
        const uint32_t cw = __ldg(R + 10 + (wi >> 2));
        below = (cw >> (8 * (wi & 3))) & 0xFFu;
        meta = mf.x;
        f = mf.y;
    }
}

// One step of a walk at state st on symbol c (c >= sigma or past the limit
// ends it).  Returns 0 = moved to st, 1 = stopped at st (output of st),
// 2 = stopped on a merged leaf (output leaf_fin[st]).
// bmask: META_BASE_MASK, or (1 << psh) - 1 for packed records.
__device__ __forceinline__ int take_step(uint32_t sigma, uint32_t c, uint32_t word,
                                         uint32_t below, uint32_t meta, uint32_t &st,
                                         uint32_t bmask = META_BASE_MASK) {
    const uint32_t bit = c & 31;
    if (c >= sigma || !((word >> bit) & 1u)) return 1;
    const uint32_t rank = below + (uint32_t)__popc(word & ((1u << bit) - 1u));
    st = (meta & bmask) + rank;
    return (meta & META_ALL_LEAF) ? 2 : 0;
}

// Output of a record in the packed format: its bit in fbc, then its rank
// among the records with an output.  The second load is taken whatever the
// bit (clamped to the array), so that a batch of these overlaps.
__device__ __forceinline__ uint32_t pk_fin(const MatchParams &P, uint32_t r) {
    const uint2 b = __ldg(reinterpret_cast<const uint2 *>(P.T.fbc) + (r >> 5));
    const uint32_t bit = r & 31;
    const uint32_t i = b.y + (uint32_t)__popc(b.x & ((1u << bit) - 1u));
    const uint32_t last = P.T.n_fvals - 1u;
    const uint32_t v = __ldg(P.T.fvals + (i < last ? i : last));
    return ((b.x >> bit) & 1u) ? v : 0u;
}

// Output of record r when the walk stops there: the separate array (W == 1),
// the packed format's rank lookup when its meta word says it has one
// (W == 0), or the word loaded with the record (f, wider records).
template <int W>
__device__ __forceinline__ uint32_t rec_fin(const MatchParams &P, uint32_t r, uint32_t f,
                                            uint32_t meta) {
    if (W == 0) return (meta & PK_FIN) ? pk_fin(P, (uint32_t)chk(P, r, P.T.n_rec)) : 0u;
    if (W == 3) return __ldg(P.T.dfin + chk(P, r, P.T.n_rec));
    if (W == 1) return __ldg(P.T.fin + chk(P, r, P.T.n_rec));
    return f;
}

// Walk of the merged trie (reduction step 2 of Section 3.2) from tree record
// s at slice offset q: records with META_IND reach their children through
// ind[]; below the last tree record u the walk counts its depth d and packs
// the symbols taken, and a stop there takes its output from the side table
// under (u, d, symbols), absent meaning none.  Every walk that reaches an
// indirect record, or a prefix entry whose state is a tail record, ends
// here; they are the walks that come within three levels of a pattern's
// end.
template <int W>
__device__ __noinline__ uint32_t dag_walk(const MatchParams *PP, uint32_t s, uint32_t q,
                                          uint32_t lim, uint32_t unit) {
    const MatchParams &P = *PP;
    const uint64_t ub = (uint64_t)unit << SLICE_SHIFT;
    const uint32_t sigma = P.T.sigma, n_upper = P.T.n_upper, bps = P.T.bps, psh = P.T.pk_shift;
    // packed records mark the indirect ones with the all-leaf flag
    const uint32_t bmask = W == 0 ? (1u << psh) - 1u : META_BASE_MASK;
    const uint32_t indf = W == 0 ? META_ALL_LEAF : META_IND;
    uint32_t u = s, d = 0, tp = 0, f = 0, meta = 0;
    for (;;) {
        const uint32_t c = q < lim ? (uint32_t)__ldg(P.in + chk(P, ub + q, P.n)) : 0x100u;
        uint32_t word, below;
        load_step<W>(P.T.rec, (uint32_t)chk(P, s, P.T.n_rec), c, word, below, meta, f, psh);
        const uint32_t bit = c & 31;
        if (c >= sigma || !((word >> bit) & 1u)) break;
        const uint32_t i = (meta & bmask) + below + (uint32_t)__popc(word & ((1u << bit) - 1u));
        s = (meta & indf) ? __ldg(P.T.ind + chk(P, i, P.T.ind_words)) : i;
        q++;
        if (s < n_upper) {
            u = s;
            d = 0;
            tp = 0;
        } else {
            tp |= c << (bps * d);
            d++;
        }
    }
    if (s < n_upper) return rec_fin<W>(P, s, f, meta);
    const uint64_t key = dag_side_key(u, d, tp);
    const uint32_t n = P.T.side_slots;
    uint64_t h = dag_side_slot(key, n);
    // a fifth of the slots at least are empty, so a probe meets the key or a hole
    for (uint32_t i = 0; i < n; i++) {
        const uint64_t kk = __ldg(reinterpret_cast<const unsigned long long *>(P.T.side_keys) + h);
        if (kk == key) return __ldg(P.T.side_vals + h);
        if (kk == DAG_SIDE_EMPTY) break;
        h = h + 1 == n ? 0 : h + 1;
    }
    return 0;
}

// Resolves queue entries [e0, e0 + 32 * walks_per_lane(W)): a few rounds
// with every lane advancing its walks together (most walks end within one or
// two levels), then the walks still running are compacted one per lane, so
// the long ones no longer cost the instructions of a full batch per level.
// Entry e's output (fin of the state its walk stops at) replaces q[e].x.
template <int W, int VAR>
__device__ __forceinline__ void resolve_pass(const MatchParams &P, QEntry *q, uint32_t n,
                                             uint32_t e0, const uint32_t *Fs, const uint32_t *Cs,
                                             const uint32_t *Es, uint32_t *tail,
                                             uint32_t lane) {
    constexpr int QU = pass_walks(W, VAR);
    constexpr int LOCK_ROUNDS = 3;
    constexpr bool DAG = (VAR & VAR_MERGED) != 0;
    const uint32_t sigma = P.T.sigma, k = P.k, rep = P.rep_log2;
    const uint32_t psh = W == 3 ? P.T.sigma : P.T.pk_shift;
    const uint32_t bmask = W == 0 ? (1u << psh) - 1u : META_BASE_MASK;
    const uint32_t *__restrict__ rec = P.T.rec;
    uint32_t st[QU], qq[QU], lim[QU], fin[QU], unit[QU];
    // -1 idle, 0 walking, 1 stopped at st, 2 stopped on merged leaf st, 3 done,
    // 4 to finish on the merged trie's slow path from tree record st at qq
    int state[QU];
    // ---- phase A: prefix entries (independent loads for all entries)
#pragma unroll
    for (int u = 0; u < QU; u++) {
        const uint32_t e = e0 + lane + 32u * u;
        state[u] = -1;
        fin[u] = 0;
        st[u] = 0;
        qq[u] = 0;
        lim[u] = 0;
        unit[u] = 0xFFFFFFFFu;
        if (e < n) {
            const QEntry en = q[e];
            unit[u] = en.unit;
            lim[u] = en.lim;
            const uint32_t p = en.pos & 0x3FFu;
            if (en.x == ROOT_X) {
                state[u] = 0;
                qq[u] = p;
            } else {
                const uint32_t xx = (uint32_t)chk(P, en.x, 1ull << (k * P.T.bps));
                const uint32_t r = (uint32_t)chk(P, prefix_rank(Fs, rep, Cs, P.c_shift, xx),
                                                 P.T.n_e[k]);
                const uint32_t ev = (VAR & 7) == VAR_FE ? Es[r] : __ldg(P.E + r);
                qq[u] = p + k;
                if (ev & D_CONT) {
                    state[u] = 0;
                    st[u] = ev & D_VAL_MASK;
                    if (DAG && (ev & D_TAIL)) {
                        // a tail record of the merged trie: walk again from
                        // the last tree record, d symbols back
                        state[u] = 4;
                        st[u] = ev & D_TAIL_REC;
                        qq[u] -= (ev >> D_TAIL_SHIFT) & 3u;
                    }
                } else {
                    state[u] = 3;
                    fin[u] = ev;
                }
            }
        }
    }
    // ---- phase B: lockstep rounds
    for (int round = 0; round < LOCK_ROUNDS; round++) {
        bool any = false;
#pragma unroll
        for (int u = 0; u < QU; u++) any |= state[u] == 0;
        if (!__any_sync(0xFFFFFFFFu, any)) break;
        uint32_t c[QU], wd[QU], bl[QU], mt[QU], f1[QU];
#pragma unroll
        for (int u = 0; u < QU; u++) {
            if (state[u] != 0) continue;
            const uint64_t ab = ((uint64_t)unit[u] << SLICE_SHIFT) + qq[u];
            c[u] = qq[u] < lim[u] ? (uint32_t)__ldg(P.in + chk(P, ab, P.n)) : 0x100u;
        }
#pragma unroll
        for (int u = 0; u < QU; u++) {
            if (state[u] != 0) continue;
            load_step<W>(rec, (uint32_t)chk(P, st[u], P.T.n_rec), c[u], wd[u], bl[u], mt[u], f1[u],
                         psh);
        }
#pragma unroll
        for (int u = 0; u < QU; u++) {
            if (state[u] != 0) continue;
            const uint32_t cur = st[u];
            const int r = take_step(sigma, c[u], wd[u], bl[u], mt[u], st[u], bmask);
            if (r == 0) {
                qq[u]++;
            } else if (r == 1) {
                // the output: loaded after phase C (separate arrays), known
                // now (a packed record without one, or the wider records)
                if (W == 0 && !(mt[u] & PK_FIN)) {
                    fin[u] = 0;
                    state[u] = 3;
                } else {
                    constexpr bool sep = W <= 1 || W == 3;  // outputs in their own array
                    if (sep) st[u] = cur;
                    else fin[u] = f1[u];
                    state[u] = sep ? 1 : 3;
                }
            } else if (DAG) {
                st[u] = cur;
                state[u] = 4;
            } else {
                state[u] = 2;
            }
        }
    }
    // ---- phase C: compact the walks still running, one per lane
    uint32_t nt = 0;
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int u = 0; u < QU; u++) {
        const bool w = state[u] == 0;
        const uint32_t b = __ballot_sync(0xFFFFFFFFu, w);
        if (w) {
            // entry index (7 bits) and position; the state goes to the entry
            const uint32_t t = nt + __popc(b & lt), e = e0 + lane + 32u * u;
            tail[t] = (e - e0) | (qq[u] << 7);
            q[e].x = st[u];
        }
        nt += __popc(b);
    }
    __syncwarp();
    // ---- outputs of the walks that ended in phases A and B: loaded now,
    // stored after phase D so the loads' latency overlaps the long walks
#pragma unroll
    for (int u = 0; u < QU; u++) {
        if (state[u] == 1) fin[u] = rec_fin<W>(P, st[u], 0, PK_FIN);
        else if (state[u] == 2) fin[u] = __ldg(P.T.leaf_fin + chk(P, st[u], P.T.leaf_words));
    }
    // ---- phase D: the long walks, one per lane
    for (uint32_t t0 = 0; t0 < nt; t0 += 32) {
        const uint32_t t = t0 + lane;
        if (t < nt) {
            const uint32_t e = e0 + (tail[t] & 0x7Fu);
            uint32_t q1 = tail[t] >> 7;
            const QEntry en = q[e];
            uint32_t s1 = en.x;
            const uint64_t ub = (uint64_t)en.unit << SLICE_SHIFT;
            uint32_t f = 0;
            // Each round fetches TS consecutive records from the current state
            // and the next TS symbols; along a single-child chain (placed in
            // consecutive records) a round advances up to TS levels.
            constexpr int TS = (W == 8 || W == 2) ? 4 : 8;  // (wider records: fewer per round, no spills)
            const uint32_t n_rec = P.T.n_rec;
            bool done = false;
            while (!done) {
                uint32_t c[TS], wd[TS], bl[TS], mt[TS], f1[TS];
#pragma unroll
                for (int i = 0; i < TS; i++) {
                    c[i] = q1 + i < en.lim ? (uint32_t)__ldg(P.in + chk(P, ub + q1 + i, P.n)) : 0x100u;
                    if (i == 0 || s1 + i < n_rec) {
                        load_step<W>(rec, (uint32_t)chk(P, s1 + i, n_rec), c[i], wd[i], bl[i],
                                     mt[i], f1[i], psh);
                    } else {
                        wd[i] = bl[i] = mt[i] = f1[i] = 0;
                    }
                }
#pragma unroll
                for (int i = 0; i < TS; i++) {
                    // state s1 + i holds the data of block entry i while the
                    // walk stays on the consecutive chain
                    uint32_t nx = 0;
                    const uint32_t cur = s1 + i;
                    const int r = take_step(sigma, c[i], wd[i], bl[i], mt[i], nx, bmask);
                    if (r == 1) {
                        f = rec_fin<W>(P, cur, f1[i], mt[i]);
                        done = true;
                        break;
                    }
                    if (r == 2) {
                        if (DAG) {
                            // finished on the merged trie's slow path below,
                            // from record cur at q1 + i
                            tail[t] = (tail[t] & 0x7Fu) | ((q1 + i) << 7);
                            f = DAG_PENDING | cur;
                        } else {
                            f = __ldg(P.T.leaf_fin + chk(P, nx, P.T.leaf_words));
                        }
                        done = true;
                        break;
                    }
                    if (i + 1 < TS && nx == cur + 1) continue;
                    s1 = nx;
                    q1 += i + 1;
                    break;
                }
            }
            q[e].x = f;
        }
    }
    // ---- the merged trie's slow path, out of the loops above: walks that
    // reached an indirect record (phase B and D) or a prefix entry on a tail
    // record (phase A)
    if (DAG) {
        __syncwarp();
        for (uint32_t t = lane; t < nt; t += 32) {
            const uint32_t e = e0 + (tail[t] & 0x7Fu);
            const QEntry en = q[e];
            if (en.x & DAG_PENDING)
                q[e].x = dag_walk<W>(&P, en.x & ~DAG_PENDING, tail[t] >> 7, en.lim, en.unit);
        }
#pragma unroll
        for (int u = 0; u < QU; u++)
            if (state[u] == 4) fin[u] = dag_walk<W>(&P, st[u], qq[u], lim[u], unit[u]);
    }
#pragma unroll
    for (int u = 0; u < QU; u++)
        if (state[u] >= 1) q[e0 + lane + 32u * u].x = fin[u];
    __syncwarp();
}

template <int W, int VAR>
__device__ __forceinline__ void resolve_batch_inl(const MatchParams &P, QEntry *q, uint32_t n,
                                                  const uint32_t *Fs, const uint32_t *Cs,
                                                  const uint32_t *Es, uint32_t lane) {
    constexpr uint32_t per = 32u * pass_walks(W, VAR);
    // the tail list lives behind the queue entries of this warp
    uint32_t *tail = reinterpret_cast<uint32_t *>(q + QCAP);
    for (uint32_t e0 = 0; e0 < n; e0 += per)
        resolve_pass<W, VAR>(P, q, n, e0, Fs, Cs, Es, tail, lane);
    __syncwarp();
}

template <int W, int VAR>
__device__ __forceinline__ void resolve_batch(const MatchParams &P, QEntry *q, uint32_t n,
                                              const uint32_t *Fs, const uint32_t *Cs,
                                              const uint32_t *Es, uint32_t lane) {
    resolve_batch_inl<W, VAR>(P, q, n, Fs, Cs, Es, lane);
}

// Filter of one slice by one warp.  Fills the survivor masks of the lane's
// 16 positions and their walk limits (relative to the slice start).  The
// first stage tests the k-symbol prefix index against the prefix bitmap F_k,
// or, with the gram filter, the next g symbols against G.
template <int BPS>
__device__ __forceinline__ void filter_slice(const MatchParams &P, const uint8_t *sb,
                                             uint32_t staged, uint32_t valid, uint32_t rem,
                                             uint32_t lima, uint32_t limb, bool general_lims,
                                             const uint64_t *__restrict__ gseg, uint64_t ustart,
                                             const uint32_t *Fs, const uint32_t *Gs,
                                             const uint32_t *Bs, uint32_t lane, uint32_t &surv,
                                             uint32_t &rootm, uint32_t (&bs)[BPS + 1]) {
    const uint32_t p0 = lane * QBPT;
    const uint32_t k = P.kf, rep = P.rep_log2;
    surv = 0;
    rootm = 0;
    if (p0 >= valid) {
#pragma unroll
        for (int w = 0; w <= BPS; w++) bs[w] = 0;
        return;
    }
    const uint4 a = *reinterpret_cast<const uint4 *>(sb + p0);
    const uint4 b = *reinterpret_cast<const uint4 *>(sb + p0 + 16);
    const uint32_t x[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    pack_symbols<BPS>(x, bs);
    if (P.tbl_b_words) {
        // prefix bytes: one byte per index, nonzero when the index has an entry
        const uint32_t kmask = (1u << (BPS * k)) - 1u;
        const uint8_t *Bb = reinterpret_cast<const uint8_t *>(Bs);
#pragma unroll
        for (int j = 0; j < QBPT; j++)
            if (Bb[chk(P, symbols_at<BPS>(bs, j) & kmask, P.tbl_b_words * 4ull)]) surv |= 1u << j;
    } else if (P.tbl_g_words == 0) {
        const uint32_t kmask = (1u << (BPS * k)) - 1u;  // k * BPS >= 5
        // Byte offset of the word of index t in copy `copy`:
        // ((((t & kmask) >> 5) << rep) | copy) * 4.  Rotating t right by
        // 3 - rep (left by rep - 3) puts the word bits at rep + 2 and
        // everything else (the bit number, the symbols above the window, the
        // wrapped bits) outside wmask, so one rotate and one and-or give it.
        const uint32_t ramt = (3u - rep) & 31u;
        const uint32_t wmask = (kmask >> 5) << (rep + 2);
        const uint32_t c4 = (lane & ((1u << rep) - 1u)) << 2;
        const uint8_t *Fb = reinterpret_cast<const uint8_t *>(Fs);
        // Each test rotates bit t & 31 of its word to bit 0 and shifts it in
        // at the top of acc (one funnel shift): position j ends at bit 16 + j.
        uint32_t acc = 0;
#pragma unroll
        for (int j = 0; j < QBPT; j++) {
            const uint32_t t = symbols_at<BPS>(bs, j);
            const uint32_t w = *reinterpret_cast<const uint32_t *>(
                Fb + chk(P, (__funnelshift_r(t, t, ramt) & wmask) | c4, P.tbl_words * 4ull));
            acc = __funnelshift_r(acc, __funnelshift_r(w, w, t), 1);
        }
        surv = acc >> (32 - QBPT);
    } else {
        // gram filter: y = t * gram_mul(g * BPS) for the window t (its bits
        // above the g symbols drop out of y); word = top hbw bits of y, bit
        // = t & 31 (table.h), copies interleaved
        const uint32_t gm = gram_mul(BPS * k);
        const uint32_t gr = P.g_rep, hbw = P.g_hb - 5;
        const uint32_t gsh = 30u - hbw - gr;  // y >> gsh puts the word at bit gr + 2
        const uint32_t gwm = ((1u << hbw) - 1u) << (gr + 2);
        const uint32_t c4 = (lane & ((1u << gr) - 1u)) << 2;
        const uint8_t *Gb = reinterpret_cast<const uint8_t *>(Gs);
        uint32_t acc = 0;  // as for the bitmap: position j ends at bit 16 + j
#pragma unroll
        for (int j = 0; j < QBPT; j++) {
            const uint32_t t = symbols_at<BPS>(bs, j);
            const uint32_t y = t * gm;
            const uint32_t w = *reinterpret_cast<const uint32_t *>(
                Gb + chk(P, ((y >> gsh) & gwm) | c4, P.tbl_g_words * 4ull));
            acc = __funnelshift_r(acc, __funnelshift_r(w, w, t), 1);  // bit t & 31
        }
        surv = acc >> (32 - QBPT);
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
    // every position's window is available (the window limits are exact
    // only when the slice's segment ends fit the lane's window)
    if (!general_lims && p0 + QBPT - 1 + k <= lim0 && p0 + QBPT <= valid && badb == 0) return;
    // fv: positions whose whole window lies in their segment and the stage;
    // ex: positions inside their segment (the others start no walk)
    uint32_t fv = 0, ex = 0;
    if (!general_lims) {
        // positions before lima end at lima, the others at limb: each set is
        // a run of low bits, so the masks come from a few compares
        auto below = [&](uint32_t x) -> uint32_t {  // positions p0 + j < x
            const uint32_t n = x > p0 ? (x - p0 < (uint32_t)QBPT ? x - p0 : (uint32_t)QBPT) : 0u;
            return (1u << n) - 1u;
        };
        const uint32_t in_a = below(lima), vm = below(valid);
        const uint32_t la = lima < staged ? lima : staged, lb = limb < staged ? limb : staged;
        const uint32_t fa = la >= k ? below(la - k + 1) : 0u;  // p + k <= la
        const uint32_t fb = lb >= k ? below(lb - k + 1) : 0u;
        ex = (in_a | below(limb)) & vm;
        fv = ((fa & in_a) | (fb & ~in_a)) & vm;
    } else {
#pragma unroll 1
        for (int j = 0; j < QBPT; j++) {
            const uint32_t p = p0 + j;
            if (p >= valid) break;
            uint32_t lo = 1, hi = P.n_seg;
            const uint64_t ap = ustart + p;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (__ldg(gseg + mid) > ap) hi = mid; else lo = mid + 1;
            }
            const uint64_t e = __ldg(gseg + lo);
            const uint64_t r = e > ustart ? e - ustart : 0;
            const uint32_t lj = r < rem ? (uint32_t)r : rem;
            if (lj > p) ex |= 1u << j;
            const uint32_t lw = lj < staged ? lj : staged;
            if (p + k <= lw) fv |= 1u << j;
        }
    }
    if (badb) {
        // windows holding a byte outside the packed symbol range
        uint32_t bw = 0;
        for (uint32_t t = 0; t < k; t++) bw |= badb >> t;
        fv &= ~bw;
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

// Symbols j.. of the lane's packed bit string for a run-time j (survivors
// only): the words it can start in are few, so a select chain replaces an
// indexed register access.
template <int BPS>
__device__ __forceinline__ uint32_t symbols_dyn(const uint32_t (&bs)[BPS + 1], uint32_t j) {
    constexpr int WMAX = (15 * BPS) >> 5;
    const uint32_t bit = BPS * j, w = bit >> 5;
    uint32_t lo = bs[0], hi = bs[1];
#pragma unroll
    for (int i = 1; i <= WMAX; i++)
        if (w == (uint32_t)i) {
            lo = bs[i];
            hi = bs[i + 1];
        }
    return __funnelshift_r(lo, hi, bit & 31);
}

// Second on-chip stage for one survivor.  With prefix bytes as the first
// stage, the next symbol's bucket must be set in the index's byte (or the
// byte is 0xFF).  With the gram filter as the first stage, the prefix index
// must be set in F_k (the filter may let other positions through).  With
// child masks, a survivor whose depth-k state
// reports nothing and has no child on the next symbol (read from the staged
// slice) stops there silently and is dropped: an entry that reports output
// has an all-ones mask and is kept whatever follows; a byte outside the
// alphabet ends every other walk.  A survivor whose next symbol is not at
// hand passes the mask test.
__device__ __forceinline__ bool mask_keep(const MatchParams &P, uint32_t x, uint32_t p,
                                          uint32_t lim, const uint8_t *sb, uint32_t staged,
                                          const uint32_t *Fs, const uint32_t *Cs,
                                          const uint32_t *Ms) {
    if (P.tbl_b_words) {
        // the prefix byte's bucket of the next symbol (shared memory offset 0)
        const uint32_t qb = p + P.k, sigma = P.T.sigma;
        if (qb < staged && qb < lim) {
            extern __shared__ __align__(128) uint8_t smem[];
            const uint32_t v = smem[chk(P, x, P.tbl_b_words * 4ull)], cs = sb[chk(P, qb, QSTAGE)];
            if (v != 0xFFu && (cs >= sigma || !((v >> byte_bucket(cs, sigma)) & 1u))) return false;
        }
    }
    if (P.tbl_g_words) {
        const uint32_t fwd = Fs[chk(P, (x >> 5) << P.rep_log2, P.tbl_words)];
        if (!((fwd >> (x & 31)) & 1u)) return false;
    }
    if (!P.tbl_m_words) return true;
    const uint32_t qn1 = p + P.k, sigma = P.T.sigma;
    if (qn1 >= staged || qn1 >= lim) return true;
    const uint32_t r = prefix_rank(Fs, P.rep_log2, Cs, P.c_shift,
                                   (uint32_t)chk(P, x, 1ull << (P.k * P.T.bps)));
    const uint32_t mb = mask_bits(sigma), ones = mb == 32 ? 0xFFFFFFFFu : (1u << mb) - 1u;
    const uint32_t mi = (uint32_t)chk(P, mb == 32 ? r : (r * mb) >> 5, P.tbl_m_words);
    const uint32_t mr = mb == 32 ? Ms[mi] : (Ms[mi] >> ((r * mb) & 31)) & ones;
    const uint32_t cs = sb[chk(P, qn1, QSTAGE)];
    return cs < sigma ? ((mr >> child_hash(cs, sigma)) & 1u) != 0 : mr == ones;
}

// Hands a queue of whole slices (q[0, qn), its last entry ending a slice)
// to the resolver kernel when the plan has one and its buffers have room:
// the entries are copied to the next free range of P.defer and a batch
// {first, n} is recorded (an empty batch when the entries do not fit).
// Returns true when the queue was handed over; the caller resolves it
// itself otherwise.
__device__ __forceinline__ bool defer_queue(const MatchParams &P, const QEntry *q, uint32_t qn,
                                            uint32_t lane) {
    if (!P.defer || qn == 0) return false;
    uint32_t eb = 0, bb = 0;
    if (lane == 0) {
        eb = atomicAdd(&P.hdr->defer_entries, qn);
        bb = atomicAdd(&P.hdr->defer_batches, 1u);
    }
    eb = __shfl_sync(0xFFFFFFFFu, eb, 0);
    bb = __shfl_sync(0xFFFFFFFFu, bb, 0);
    const bool room = eb + qn <= P.defer_cap && eb + qn >= eb;
    if (bb < P.dbatch_cap && lane == 0) P.dbatch[bb] = make_uint2(eb, room ? qn : 0u);
    if (!room || bb >= P.dbatch_cap) return false;
    for (uint32_t i = lane; i < qn; i += 32)
        P.defer[chk(P, eb + i, P.defer_cap)] = *reinterpret_cast<const uint4 *>(&q[chk(P, i, QCAP)]);
    __syncwarp();
    return true;
}

// Record-mode flush: resolve the queue, then keep a record (position, fin)
// for each matched survivor, ranked among its slice's matched survivors (the
// slice's entries are contiguous in the queue and resolve in one batch).
// The last entry of each slice publishes the slice's record count; slices
// with more matches than their record space (P.unit_cap) go to the emit pass.
//
// A slice may also span batches (a kernel that resolves a slice with more
// survivors than its queue holds in queue-sized chunks): the entries of
// slice `carry_unit` then rank after the `carry` records of its earlier
// batches, and when the batch's last entry is not its slice's last, that
// slice and its records so far are returned in carry_unit / carry for the
// next batch (carry_unit = UNIT_OVF when no slice continues).
template <int W, int VAR>
__device__ __forceinline__ void flush_records_c(const MatchParams &P, QEntry *q, uint32_t n,
                                                const uint32_t *Fs, const uint32_t *Cs,
                                                const uint32_t *Es, uint32_t lane,
                                                uint32_t &carry_unit, uint32_t &carry) {
    if (n == 0) return;
    resolve_batch<W, VAR>(P, q, n, Fs, Cs, Es, lane);
    uint32_t fin[QU], pos[QU], unit[QU];
#pragma unroll
    for (int u = 0; u < QU; u++) {
        const uint32_t e = lane + 32u * u;
        unit[u] = 0xFFFFFFFFu;
        fin[u] = 0;
        pos[u] = 0;
        if (e < n) {
            unit[u] = q[e].unit;
            pos[u] = q[e].pos;
            fin[u] = q[e].x;
        }
    }
    __syncwarp();
    // exclusive count of matched entries before each entry of the batch
    uint32_t pre[QU], carry_in = 0;
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int u = 0; u < QU; u++) {
        const uint32_t b = __ballot_sync(0xFFFFFFFFu, fin[u] != 0);
        pre[u] = carry_in + __popc(b & lt);
        carry_in += __popc(b);
    }
#pragma unroll
    for (int u = 0; u < QU; u++)
        if (unit[u] != 0xFFFFFFFFu) q[lane + 32u * u].x = pre[u];
    __syncwarp();
    const uint32_t cap = P.unit_cap;
    uint32_t cu = UNIT_OVF, cc = 0;
#pragma unroll
    for (int u = 0; u < QU; u++) {
        if (unit[u] == 0xFFFFFFFFu) continue;
        const uint32_t e = lane + 32u * u;
        const uint32_t p = pos[u] & 0x3FFu, slot = (pos[u] >> 10) & 0xFFu;
        const bool last = (pos[u] & LAST_FLAG) != 0;
        const uint32_t base = q[e - slot].x;
        const uint32_t rank = pre[u] - base + (unit[u] == carry_unit ? carry : 0u);
        const uint32_t uu = (uint32_t)chk(P, unit[u], P.n_tiles);
        if (fin[u]) {
            if (rank < cap) P.recs[(size_t)uu * cap + rank] = ((uint64_t)p << 32) | fin[u];
            atomicAdd((unsigned long long *)(P.tile_k + uu), (unsigned long long)fin_len_c(P, fin[u]));
        }
        const uint32_t m = rank + (fin[u] ? 1u : 0u);
        if (last) {
            if (m > cap) {
                P.tile_m[uu] = UNIT_OVF;
                P.ovf_list[chk(P, atomicAdd(&P.hdr->ovf_count, 1u), P.n_tiles)] = uu;
            } else {
                P.tile_m[uu] = m;
            }
        } else if (e == n - 1) {
            cu = unit[u];
            cc = m;
        }
    }
    carry_unit = __shfl_sync(0xFFFFFFFFu, cu, (n - 1) & 31u);
    carry = __shfl_sync(0xFFFFFFFFu, cc, (n - 1) & 31u);
    __syncwarp();
}

template <int W, int VAR>
__device__ __forceinline__ void flush_records(const MatchParams &P, QEntry *q, uint32_t n,
                                              const uint32_t *Fs, const uint32_t *Cs,
                                              const uint32_t *Es, uint32_t lane) {
    uint32_t cu = UNIT_OVF, cc = 0;
    flush_records_c<W, VAR>(P, q, n, Fs, Cs, Es, lane, cu, cc);
}

// Appends the candidates of the lanes set in `lanes` to the queue after the
// second on-chip stage (mask_keep), in position order.  Entry fields: the
// slice, the position, the slot among the slice's appended survivors and,
// on the last one, LAST_FLAG; the prefix index (or ROOT_X); the walk limit.
// Three ways, by the slice's candidates:
//   * at most two per lane: every lane tests and writes its own;
//   * at most QCAP: every lane parks its own candidates in the warp's
//     scratch (the long-walk buffer, idle here), then lane i takes candidate
//     i of each group of 32 for the test and the queue write;
//   * more: candidate i of each group of 32 goes to lane i, which finds the
//     owning lane by a shuffle search over the lanes' exclusive counts and
//     the position in that lane's mask by __fns.
// Returns AP_DONE (qn advanced), AP_FLUSH (the queue must be resolved first:
// the caller flushes q[0, qn), moves the slice's st.kept entries at q[qn..]
// to the front and calls again with qn = 0; the call resumes where it
// stopped) or AP_OVER (more than a whole queue survives; qn is 0).
enum { AP_DONE = 0, AP_FLUSH = 1, AP_OVER = 2 };
struct AppendState {
    uint32_t base;  // next group of 32 candidates (dense slices)
    uint32_t kept;  // entries of this slice already in the queue
    bool flagged;   // LAST_FLAG written
};

template <int BPS>
__device__ __forceinline__ int append_slice(const MatchParams &P, QEntry *q, uint32_t qn,
                                            AppendState &st, uint32_t cand, uint32_t rootm,
                                            uint32_t lanes, const uint32_t (&bs)[BPS + 1],
                                            const uint8_t *sb, uint32_t staged, uint32_t unit,
                                            uint32_t lima, uint32_t limb, bool general_lims,
                                            uint64_t ustart, uint32_t rem, const uint32_t *Fs,
                                            const uint32_t *Cs, const uint32_t *Ms, uint32_t lane) {
    const uint32_t m = ((lanes >> lane) & 1u) ? cand : 0u;
    const uint32_t c = __popc(m);
    const uint32_t k = P.k, kmask = (1u << (BPS * k)) - 1u;
    const bool stage2 = P.tbl_m_words != 0 || P.tbl_g_words != 0 || P.tbl_b_words != 0;
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t p0 = lane * QBPT;
    auto entry = [&](uint32_t p, uint32_t x, uint32_t lim, uint32_t slot, bool last) {
        QEntry en;
        en.unit = unit;
        en.pos = p | (slot << 10) | (last ? LAST_FLAG : 0u);
        en.x = x;
        en.lim = lim;
        return en;
    };

    if (__reduce_max_sync(0xFFFFFFFFu, c) <= 2u) {
        // sparse: every lane tests and writes its own (at most two) candidates
        uint32_t keepm = m;
        if (stage2) {
            uint32_t mm = m & ~rootm;
            while (mm) {
                const uint32_t j = __ffs(mm) - 1;
                mm &= mm - 1;
                const uint32_t p = p0 + j;
                if (!mask_keep(P, symbols_dyn<BPS>(bs, j) & kmask, p,
                               lim_of(P, p, lima, limb, general_lims, ustart, rem), sb, staged,
                               Fs, Cs, Ms))
                    keepm &= ~(1u << j);
            }
        }
        const uint32_t kc = __popc(keepm);
        const uint32_t b1 = __ballot_sync(0xFFFFFFFFu, kc >= 1u);
        const uint32_t b2 = __ballot_sync(0xFFFFFFFFu, kc >= 2u);
        const uint32_t kept = __popc(b1) + __popc(b2);
        if (qn + kept > (uint32_t)QCAP) return qn ? AP_FLUSH : AP_OVER;
        uint32_t o = __popc(b1 & lt) + __popc(b2 & lt), mm = keepm;
        while (mm) {
            const uint32_t j = __ffs(mm) - 1;
            mm &= mm - 1;
            const uint32_t p = p0 + j;
            const uint32_t x = ((rootm >> j) & 1u) ? ROOT_X : (symbols_dyn<BPS>(bs, j) & kmask);
            q[qn + o] = entry(p, x, lim_of(P, p, lima, limb, general_lims, ustart, rem), o,
                              o + 1 == kept);
            o++;
        }
        __syncwarp();
        st.kept = kept;
        return AP_DONE;
    }

    uint32_t inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t nb = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= (uint32_t)o) inc += nb;
    }
    const uint32_t tot = __shfl_sync(0xFFFFFFFFu, inc, 31);
    const uint32_t excl = inc - c;
    if (tot <= (uint32_t)QCAP) {
        // Each lane parks its candidates in the scratch as one word: position
        // (9 bits), prefix index (21 bits; narrow symbols only, wide ones
        // are re-read from the stage), root flag (bit 31).  The scratch is
        // rebuilt when the call resumes after a flush, which reuses it.
        uint32_t *scratch = reinterpret_cast<uint32_t *>(q + QCAP);  // QCAP words
        uint32_t o = excl, mm = m;
        while (mm) {
            const uint32_t j = __ffs(mm) - 1;
            mm &= mm - 1;
            const uint32_t root = (rootm >> j) & 1u;
            const uint32_t x = BPS <= 5 && !root ? (symbols_dyn<BPS>(bs, j) & kmask) : 0u;
            scratch[o++] = (p0 + j) | (x << 9) | (root << 31);
        }
        __syncwarp();
        for (; st.base < tot; st.base += 32) {
            const uint32_t i = st.base + lane;
            const bool valid = i < tot;
            const uint32_t e = valid ? scratch[i] : 0u;
            const uint32_t p = e & 511u;
            // the owning lane's segment ends
            const uint32_t laL = __shfl_sync(0xFFFFFFFFu, lima, p / QBPT);
            const uint32_t lbL = __shfl_sync(0xFFFFFFFFu, limb, p / QBPT);
            uint32_t x = ROOT_X, lim = 0;
            bool keep = false;
            if (valid) {
                lim = lim_of(P, p, laL, lbL, general_lims, ustart, rem);
                keep = true;
                if (!(e >> 31)) {
                    if (BPS <= 5) {
                        x = (e >> 9) & 0x1FFFFFu;
                    } else {
                        // k <= 3 symbols of the window, first symbol lowest
                        x = 0;
                        for (uint32_t t = 0; t < k; t++)
                            x |= ((uint32_t)sb[p + t] & ((1u << BPS) - 1u)) << (BPS * t);
                    }
                    if (stage2) keep = mask_keep(P, x, p, lim, sb, staged, Fs, Cs, Ms);
                }
            }
            const uint32_t b = __ballot_sync(0xFFFFFFFFu, keep);
            const uint32_t nk = st.kept + __popc(b);
            if (qn + nk > (uint32_t)QCAP) {
                __syncwarp();
                return qn ? AP_FLUSH : AP_OVER;  // resume at this group
            }
            const uint32_t slot = st.kept + __popc(b & lt);
            const bool lastg = st.base + 32 >= tot;
            if (keep) q[qn + slot] = entry(p, x, lim, slot, lastg && slot + 1 == nk);
            if (lastg) st.flagged = b != 0;
            st.kept = nk;
        }
        __syncwarp();
        if (st.kept && !st.flagged) {
            // every candidate of the last group was dropped: flag the last kept one
            if (lane == 0) q[qn + st.kept - 1].pos |= LAST_FLAG;
            __syncwarp();
        }
        return AP_DONE;
    }

    for (; st.base < tot; st.base += 32) {
        const uint32_t base = st.base;
        const uint32_t i = base + lane;
        const bool valid = i < tot;
        // owner: the last lane whose exclusive count is <= i
        uint32_t L = 0;
#pragma unroll
        for (int s = 16; s >= 1; s >>= 1) {
            const uint32_t v = __shfl_sync(0xFFFFFFFFu, excl, L + s);
            if (v <= i) L += s;
        }
        const uint32_t exL = __shfl_sync(0xFFFFFFFFu, excl, L);
        const uint32_t mL = __shfl_sync(0xFFFFFFFFu, m, L);
        const uint32_t rL = __shfl_sync(0xFFFFFFFFu, rootm, L);
        uint32_t bsL[BPS + 1];
#pragma unroll
        for (int w = 0; w <= BPS; w++) bsL[w] = __shfl_sync(0xFFFFFFFFu, bs[w], L);
        const uint32_t laL = __shfl_sync(0xFFFFFFFFu, lima, L);
        const uint32_t lbL = __shfl_sync(0xFFFFFFFFu, limb, L);
        bool keep = false;
        uint32_t p = 0, x = ROOT_X, lim = 0;
        if (valid) {
            const uint32_t j = __fns(mL, 0, (int)(i - exL) + 1);
            p = L * QBPT + j;
            lim = lim_of(P, p, laL, lbL, general_lims, ustart, rem);
            keep = true;
            if (!((rL >> j) & 1u)) {
                x = symbols_dyn<BPS>(bsL, j) & kmask;
                keep = mask_keep(P, x, p, lim, sb, staged, Fs, Cs, Ms);
            }
        }
        const uint32_t b = __ballot_sync(0xFFFFFFFFu, keep);
        const uint32_t nk = st.kept + __popc(b);
        if (qn + nk > (uint32_t)QCAP) return qn ? AP_FLUSH : AP_OVER;  // resume at this group
        const uint32_t slot = st.kept + __popc(b & lt);
        const bool lastg = base + 32 >= tot;
        if (keep) q[qn + slot] = entry(p, x, lim, slot, lastg && slot + 1 == nk);
        if (lastg) st.flagged = b != 0;
        st.kept = nk;
    }
    __syncwarp();
    if (st.kept && !st.flagged) {
        // every candidate of the last group was dropped: flag the last kept one
        if (lane == 0) q[qn + st.kept - 1].pos |= LAST_FLAG;
        __syncwarp();
    }
    return AP_DONE;
}

// Resolves every survivor of one slice in quarters of 8 lanes (at most 128
// candidates each).  emit == 0: returns the slice's key count, and with
// record space for every position of the slice (P.unit_cap >= SLICE) also
// writes its records in position order, their number to *n_recs.  emit ==
// 1: writes the slice's keys at key_off[unit] and returns the count.
template <int W, int BPS, int VAR>
__device__ __forceinline__ uint64_t resolve_slice(const MatchParams &P, QEntry *q, uint32_t cand,
                                                  uint32_t rootm, const uint32_t (&bs)[BPS + 1],
                                                  const uint8_t *sb, uint32_t staged,
                                                  uint32_t unitid, uint32_t lima, uint32_t limb,
                                                  bool general_lims, uint64_t ustart,
                                                  uint32_t rem, const uint32_t *Fs,
                                                  const uint32_t *Cs, const uint32_t *Es,
                                                  const uint32_t *Ms, uint32_t lane, bool emit,
                                                  uint32_t *n_recs = nullptr) {
    uint64_t keys = 0;
    uint32_t nrec = 0;
    const bool records = !emit && P.unit_cap >= (uint32_t)SLICE;
    const uint64_t obase = emit ? P.key_off[unitid] : 0;
    for (int qt = 0; qt < 4; qt++) {
        AppendState ast{0u, 0u, false};
        append_slice<BPS>(P, q, 0u, ast, cand, rootm, 0xFFu << (8 * qt), bs, sb, staged, unitid,
                          lima, limb, general_lims, ustart, rem, Fs, Cs, Ms, lane);
        const uint32_t n = ast.kept;  // a quarter has at most QCAP candidates
        if (n == 0) continue;
        resolve_batch<W, VAR>(P, q, n, Fs, Cs, Es, lane);
        uint32_t fin[QU], pos[QU];
#pragma unroll
        for (int u = 0; u < QU; u++) {
            const uint32_t e = lane + 32u * u;
            fin[u] = e < n ? q[e].x : 0u;
            pos[u] = e < n ? q[e].pos : 0u;
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < QU; u++) {
            if (records) {
                // one record per matched position, ranked in position order
                const uint32_t b = __ballot_sync(0xFFFFFFFFu, fin[u] != 0);
                if (fin[u])
                    P.recs[(size_t)unitid * P.unit_cap + nrec + __popc(b & ((1u << lane) - 1u))] =
                        ((uint64_t)(pos[u] & 0x3FFu) << 32) | fin[u];
                nrec += __popc(b);
            }
            const uint32_t L = fin[u] ? fin_len_c(P, fin[u]) : 0u;
            uint32_t inc = L;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t nb = __shfl_up_sync(0xFFFFFFFFu, inc, o);
                if (lane >= (uint32_t)o) inc += nb;
            }
            const uint32_t tot = __shfl_sync(0xFFFFFFFFu, inc, 31);
            if (emit && L) {
                const uint32_t *ids = fin_ids_c(P, fin[u]);
                const uint64_t pk = (P.pos_base + ustart + (pos[u] & 0x3FFu)) << PFAC_ID_BITS;
                uint64_t o = obase + keys + inc - L;
                for (uint32_t e = 0; e < L; e++, o++)
                    if (o < P.cap) P.out[o] = pk | __ldg(ids + e);
            }
            keys += tot;
        }
        __syncwarp();
    }
    if (n_recs) *n_recs = nrec;
    return keys;
}

// EMIT == 0: the scan pass (records and key counts).  EMIT == 1: the emit
// pass over the slices listed in ovf_list.  NW warps per CTA: 16 (up to 128
// registers a thread) or 24 (up to 80; more warps to hide latency where the
// tables leave room in shared memory).  The int argument is unused (the
// launch signature is shared with the uncompressed kernel).
template <int W, int BPS, int VAR, int EMIT, int NW>
__global__ void __launch_bounds__(NW * 32, 1) k_scanq(const __grid_constant__ MatchParams P, const int) {
    constexpr uint32_t QTHREADS = NW * 32;
    constexpr bool emit = EMIT != 0;
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t n_units = emit ? *(volatile uint32_t *)&P.hdr->ovf_count : P.n_tiles;
    const uint32_t gw = blockIdx.x * NW + warp, gstride = gridDim.x * NW;
    if (blockIdx.x * NW >= n_units) return;  // the whole CTA has no unit

    uint32_t *Bs = reinterpret_cast<uint32_t *>(smem);  // prefix bytes, at offset 0
    uint32_t *Fs = Bs + P.tbl_b_words;
    uint32_t *Cs = Fs + P.tbl_words;
    uint32_t *Es = Cs + P.tbl_c_words;
    uint32_t *Ms = Es + P.tbl_e_words;
    uint32_t *Gs = Ms + P.tbl_m_words;
    WarpArea *areas = reinterpret_cast<WarpArea *>(
        smem + ((((size_t)P.tbl_b_words + P.tbl_words + P.tbl_c_words + P.tbl_e_words +
                  P.tbl_m_words + P.tbl_g_words) * 4 + 127) &
                ~(size_t)127));
    {
        const uint32_t rep = P.rep_log2;
        for (uint32_t i = threadIdx.x; i < P.tbl_words; i += QTHREADS) Fs[i] = __ldg(P.F + (i >> rep));
        for (uint32_t i = threadIdx.x; i < P.tbl_c_words; i += QTHREADS) Cs[i] = __ldg(P.C + i);
        if ((VAR & 7) == VAR_FE)
            for (uint32_t i = threadIdx.x; i < P.tbl_e_words; i += QTHREADS) Es[i] = __ldg(P.E + i);
        for (uint32_t i = threadIdx.x; i < P.tbl_m_words; i += QTHREADS) Ms[i] = __ldg(P.M + i);
        const uint32_t *bsrc = reinterpret_cast<const uint32_t *>(P.Bt);
        for (uint32_t i = threadIdx.x; i < P.tbl_b_words; i += QTHREADS) Bs[i] = __ldg(bsrc + i);
        // gram filter: word w of each copy is the OR of 2^g_fold table words
        const uint32_t gr = P.g_rep, gf = P.g_fold;
        for (uint32_t i = threadIdx.x; i < P.tbl_g_words; i += QTHREADS) {
            const uint32_t *src = P.T.G + ((size_t)(i >> gr) << gf);
            uint32_t v = 0;
            for (uint32_t f = 0; f < (1u << gf); f++) v |= __ldg(src + f);
            Gs[i] = v;
        }
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
        if (u == P.withhold_unit) return;  // testing: this stage never completes
        mbar_arrive_expect_tx(bar, bytes);
        if (bytes) bulk_g2s(A.ring[i % QRING], P.in + start, bytes, bar);
    };
    if (lane == 0)
        for (uint32_t i = 0; i < QRING; i++) issue(i);
    __syncwarp();

    const bool multi = P.n_seg > 1;
    // Segment data runs one slice ahead: while a slice is processed, the
    // offset window of the next unit and the first-offset index of the one
    // after it are in flight.
    auto load_window = [&](uint32_t sf) -> uint64_t {
        const uint32_t si = sf + lane;
        return si <= P.n_seg ? __ldg(P.seg + si) : ~0ull;
    };
    uint64_t seg_o = ~0ull;  // this lane's offset of the current unit's window
    uint32_t sf_n = 0;       // first offset index after the next unit's start
    if (multi && gw < n_units) {
        seg_o = load_window(__ldg(P.unit_seg + unit_of(0)));
        if (gw + gstride < n_units) sf_n = __ldg(P.unit_seg + unit_of(1));
    }
    uint32_t qn = 0;  // queued entries (warp-uniform)
    uint32_t i_fail = 0;
    bool failed = false;
    for (uint32_t i = 0; gw + i * gstride < n_units; i++) {
        const uint32_t u = unit_of(i);
        const uint64_t ustart = (uint64_t)u << SLICE_SHIFT;
        const uint64_t remain = P.n - ustart;
        const uint32_t rem = remain < LIM_MAX ? (uint32_t)remain : LIM_MAX;
        uint32_t valid = rem < (uint32_t)SLICE ? rem : (uint32_t)SLICE;
        {
            const uint64_t sl = P.starts_end > ustart ? P.starts_end - ustart : 0;
            if (sl < valid) valid = (uint32_t)sl;
        }
        const uint32_t staged = (rem < (uint32_t)QSTAGE ? rem : (uint32_t)QSTAGE) & ~15u;

        // segment ends of this slice: a window of 32 offsets after its start
        uint32_t lima = rem, limb = rem;
        bool general_lims = false;
        if (multi) {
            const uint64_t o = seg_o;
            seg_o = gw + (i + 1) * gstride < n_units ? load_window(sf_n) : ~0ull;
            if (gw + (i + 2) * gstride < n_units) sf_n = __ldg(P.unit_seg + unit_of(i + 2));
            uint32_t wv = LIM_MAX;
            if (o != ~0ull) {
                const uint64_t r = o > ustart ? o - ustart : 0;
                wv = r < rem ? (uint32_t)r : rem;
            }
            const uint32_t w0 = __shfl_sync(0xFFFFFFFFu, wv, 0);
            const uint32_t w1 = __shfl_sync(0xFFFFFFFFu, wv, 1);
            if (w0 >= (uint32_t)QSTAGE) {
                // no segment end inside the stage: one limit for every lane
                lima = w0 < rem ? w0 : rem;
                limb = w1 < rem ? w1 : rem;
            } else {
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
        }

        const uint32_t s = i % QRING;
        if (!mbar_wait_bounded(&A.bar[s], (i / QRING) & 1, P.wait_limit_ns)) {
            if (lane == 0) atomicOr(&P.hdr->status, ST_TIMEOUT);
            failed = true;
            i_fail = i;
            break;
        }
        const uint8_t *sb = A.ring[s];
        uint32_t surv, rootm, bs[BPS + 1];
        filter_slice<BPS>(P, sb, staged, valid, rem, lima, limb, general_lims, P.seg, ustart, Fs,
                          Gs, Bs, lane, surv, rootm, bs);
        const uint32_t cand = surv | rootm;
        const uint32_t cnt = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)__popc(cand));

        if (emit) {
            resolve_slice<W, BPS, VAR>(P, A.q, cand, rootm, bs, sb, staged, u, lima, limb,
                                       general_lims, ustart, rem, Fs, Cs, Es, Ms, lane, true);
        } else {
            // tile_m / tile_k start at zero; the slice's last entry sets its
            // record count when resolved
            int ar = AP_DONE;
            if (cnt) {
                AppendState ast{0u, 0u, false};
                for (;;) {
                    ar = append_slice<BPS>(P, A.q, qn, ast, cand, rootm, 0xFFFFFFFFu, bs, sb,
                                           staged, u, lima, limb, general_lims, ustart, rem, Fs, Cs,
                                           Ms, lane);
                    if (ar != AP_FLUSH) break;
                    // resolve the queue (or hand it over), move the slice's
                    // entries to its front
                    if (!defer_queue(P, A.q, qn, lane))
                        flush_records<W, VAR>(P, A.q, qn, Fs, Cs, Es, lane);
                    for (uint32_t e0 = 0; e0 < ast.kept; e0 += 32) {
                        const uint32_t e = e0 + lane;
                        QEntry t;
                        if (e < ast.kept) t = A.q[qn + e];
                        __syncwarp();
                        if (e < ast.kept) A.q[e] = t;
                        __syncwarp();
                    }
                    qn = 0;
                }
                if (ar == AP_DONE) qn += ast.kept;
            }
            if (ar == AP_OVER) {
                // more survivors than the (now empty) queue holds: resolved
                // now in quarters; with record space for every position the
                // records are written now, otherwise the keys are counted now
                // and written by the emit pass
                uint32_t nrec = 0;
                const uint64_t keys = resolve_slice<W, BPS, VAR>(P, A.q, cand, rootm, bs, sb,
                                                                 staged, u, lima, limb,
                                                                 general_lims, ustart, rem, Fs,
                                                                 Cs, Es, Ms, lane, false, &nrec);
                if (lane == 0) {
                    P.tile_k[u] = keys;
                    if (P.unit_cap >= (uint32_t)SLICE) {
                        P.tile_m[u] = nrec;
                    } else {
                        P.tile_m[u] = UNIT_OVF;
                        P.ovf_list[atomicAdd(&P.hdr->ovf_count, 1u)] = u;
                    }
                }
            }
        }
        // the stage is consumed: refill it with the unit QRING ahead
        __syncwarp();
        if (lane == 0) issue(i + QRING);  // every lane's reads of the stage are done
        __syncwarp();
    }
    if (!failed && !emit && !defer_queue(P, A.q, qn, lane))
        flush_records<W, VAR>(P, A.q, qn, Fs, Cs, Es, lane);
    if (failed && lane == 0) {
        // wait (bounded) for this warp's copies that may still be in flight:
        // the stages of units i_fail .. i_fail + QRING - 1
        for (uint32_t i = i_fail; i < i_fail + QRING; i++) {
            if (gw + i * gstride >= n_units) break;
            mbar_wait_bounded(&A.bar[i % QRING], (i / QRING) & 1, P.wait_limit_ns);
        }
    }
}

}  // namespace pfac

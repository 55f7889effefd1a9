// Host-side trie builder and compressor (Sections 3.1 and 3.2).
//
// Steps: validate -> sort the patterns alphabetically keeping their ids ->
// breadth-first construction (children contiguous and in symbol order) ->
// output lists per state -> leaf merge (Eq. 2) -> bitmap records with
// popcount-ranked child bases (Eq. 1) -> dense prefix lookups for the first
// levels -> one device blob uploaded on the caller's stream.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace pfac {

static thread_local int g_last_status = 0;
static thread_local char g_last_msg[512] = {0};

int set_error(int status, const char *fmt, ...) {
    g_last_status = status;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_msg, sizeof(g_last_msg), fmt, ap);
    va_end(ap);
    return status;
}

void clear_error() {
    g_last_status = 0;
    g_last_msg[0] = 0;
}

namespace {

struct BNode {
    uint32_t lo, hi;       // range of the sorted pattern list sharing the prefix
    uint32_t depth;
    uint32_t parent;
    uint32_t first_child;  // node index of the first child (valid if n_child)
    uint32_t n_child;
    uint32_t fin_lo, fin_hi;  // sorted-order range of the patterns ending here
};

struct Pat {
    const uint8_t *p;
    uint32_t len;
};

bool pat_less(const Pat &a, const Pat &b) {
    uint32_t m = a.len < b.len ? a.len : b.len;
    int c = m ? memcmp(a.p, b.p, m) : 0;
    if (c != 0) return c < 0;
    return a.len < b.len;
}

uint32_t bits_per_symbol(uint32_t sigma) {
    uint32_t b = 1;
    while ((1u << b) < sigma) b++;
    return b;
}

// Appends the sorted id list `ids` to the pool; returns its fin code.
int put_list(std::vector<uint32_t> &pool, const std::vector<uint32_t> &ids, uint32_t *code) {
    uint64_t off = pool.size();
    if (off > FIN_MAX_OFF) return -1;
    if (ids.size() < FIN_LEN_ESC) {
        pool.insert(pool.end(), ids.begin(), ids.end());
        *code = (uint32_t)(off << FIN_LEN_BITS) | (uint32_t)ids.size();
    } else {
        pool.push_back((uint32_t)ids.size());
        pool.insert(pool.end(), ids.begin(), ids.end());
        *code = (uint32_t)(off << FIN_LEN_BITS) | FIN_LEN_ESC;
    }
    return 0;
}

void get_list(const std::vector<uint32_t> &pool, uint32_t code, std::vector<uint32_t> &ids) {
    ids.clear();
    if (!code) return;
    uint32_t off = code >> FIN_LEN_BITS, len = code & FIN_LEN_ESC;
    if (len == FIN_LEN_ESC) {
        len = pool[off];
        off++;
    }
    ids.assign(pool.begin() + off, pool.begin() + off + len);
}

// sections start on 16-byte boundaries (the widest load of any of them)
inline uint64_t align16(uint64_t x) { return (x + 15) & ~15ull; }

}  // namespace
}  // namespace pfac

using namespace pfac;

extern "C" int pfac_build(const uint8_t *const *patterns, const uint32_t *lengths,
                          uint32_t n_patterns, uint32_t alphabet_size,
                          const pfac_build_opts *opts, void *cuda_stream, pfac_table **out) {
    clear_error();
    if (!out) return set_error(PFAC_EINVAL, "pfac_build: out is NULL");
    *out = nullptr;
    if (alphabet_size < 1 || alphabet_size > 256)
        return set_error(PFAC_EINVAL, "pfac_build: alphabet_size %u not in 1..256", alphabet_size);
    if (n_patterns >= (1u << PFAC_ID_BITS))
        return set_error(PFAC_EINVAL, "pfac_build: %u patterns exceed the id range", n_patterns);
    if (n_patterns && (!patterns || !lengths))
        return set_error(PFAC_EINVAL, "pfac_build: NULL pattern arrays");
    pfac_build_opts o{};
    if (opts) o = *opts;
    if (o.layout > PFAC_LAYOUT_DENSE)
        return set_error(PFAC_EINVAL, "pfac_build: unknown layout %u", o.layout);
    if (o.layout == PFAC_LAYOUT_DENSE && (o.flags & PFAC_BUILD_SUFFIX_MERGE))
        return set_error(PFAC_EINVAL, "pfac_build: PFAC_BUILD_SUFFIX_MERGE needs the compressed layout");
    const uint32_t sigma = alphabet_size;

    try {
        // ---- validate ----------------------------------------------------
        std::vector<Pat> pats(n_patterns);
        uint32_t min_len = n_patterns ? 0xFFFFFFFFu : 0, max_len = 0;
        uint64_t total = 0;
        double match_density = 0.0;
        for (uint32_t i = 0; i < n_patterns; i++) {
            uint32_t L = lengths[i];
            if (L == 0) return set_error(PFAC_EINVAL, "pfac_build: pattern %u is empty", i);
            if (L > PFAC_MAX_PATTERN_LEN)
                return set_error(PFAC_EINVAL, "pfac_build: pattern %u longer than %u", i,
                                 PFAC_MAX_PATTERN_LEN);
            if (!patterns[i]) return set_error(PFAC_EINVAL, "pfac_build: pattern %u is NULL", i);
            if (sigma < 256)
                for (uint32_t k = 0; k < L; k++)
                    if (patterns[i][k] >= sigma)
                        return set_error(PFAC_ESYMBOL,
                                         "pfac_build: pattern %u byte %u is %u >= alphabet %u", i,
                                         k, patterns[i][k], sigma);
            pats[i] = Pat{patterns[i], L};
            min_len = std::min(min_len, L);
            max_len = std::max(max_len, L);
            total += L;
            // expected matches per position of uniform text over the alphabet
            match_density += std::pow((double)sigma, -(double)L);
        }
        if (total >= 0x7FFFFFF0ull)
            return set_error(PFAC_EINVAL, "pfac_build: %llu pattern bytes exceed 2^31",
                             (unsigned long long)total);

        // ---- sort alphabetically, keeping ids (Section 3.1) --------------
        std::vector<uint32_t> order(n_patterns);
        for (uint32_t i = 0; i < n_patterns; i++) order[i] = i;
        std::sort(order.begin(), order.end(),
                  [&](uint32_t a, uint32_t b) { return pat_less(pats[a], pats[b]); });
        for (uint32_t i = 1; i < n_patterns; i++) {
            const Pat &a = pats[order[i - 1]], &b = pats[order[i]];
            if (a.len == b.len && memcmp(a.p, b.p, a.len) == 0)
                return set_error(PFAC_EDUP, "pfac_build: patterns %u and %u are equal",
                                 std::min(order[i - 1], order[i]), std::max(order[i - 1], order[i]));
        }
        // with truncation (prefix matching, Section 2.4) the trie holds every
        // pattern's first `trunc` symbols; patterns sharing them end at one node
        const uint32_t trunc = o.truncate_depth;
        auto sym_at = [&](uint32_t sorted_i, uint32_t d) { return pats[order[sorted_i]].p[d]; };
        auto len_at = [&](uint32_t sorted_i) {
            const uint32_t L = pats[order[sorted_i]].len;
            return trunc && L > trunc ? trunc : L;
        };

        // ---- breadth-first trie -----------------------------------------
        const uint32_t W = sigma <= 32 ? 1 : (sigma <= 64 ? 2 : 8);
        std::vector<BNode> nodes;
        std::vector<uint32_t> bm;  // W words per node
        nodes.reserve(total + 1);
        nodes.push_back(BNode{0, n_patterns, 0, 0, 0, 0, 0, 0});
        bm.assign(W, 0);
        for (size_t v = 0; v < nodes.size(); v++) {
            uint32_t lo = nodes[v].lo, hi = nodes[v].hi, d = nodes[v].depth;
            uint32_t i = lo;
            // the patterns equal to the prefix sort first (several only when
            // truncated)
            nodes[v].fin_lo = i;
            while (i < hi && len_at(i) == d) i++;
            nodes[v].fin_hi = i;
            while (i < hi) {
                uint8_t c = sym_at(i, d);
                uint32_t k = i;
                while (k < hi && sym_at(k, d) == c) k++;
                uint32_t idx = (uint32_t)nodes.size();
                if (nodes[v].n_child == 0) nodes[v].first_child = idx;
                nodes[v].n_child++;
                bm[v * W + (c >> 5)] |= 1u << (c & 31);
                nodes.push_back(BNode{i, k, d + 1, (uint32_t)v, 0, 0, 0, 0});
                bm.resize(bm.size() + W, 0);
                i = k;
            }
        }
        const uint64_t Q = nodes.size();
        if (Q >= 0x7FFFFFF0ull) return set_error(PFAC_EINVAL, "pfac_build: trie too large");
        // the kernels carry a state number in 30 bits
        if (Q > META_BASE_MASK)
            return set_error(PFAC_EINVAL, "pfac_build: %llu trie nodes exceed 2^30",
                             (unsigned long long)Q);

        // ---- output lists: fin(v) = fin(parent) plus v's own id ----------
        std::vector<uint32_t> fin_code(Q, 0), pool;
        std::vector<uint32_t> ids;
        uint64_t n_lists = 0;
        for (uint64_t v = 1; v < Q; v++) {
            uint32_t pc = fin_code[nodes[v].parent];
            if (nodes[v].fin_lo == nodes[v].fin_hi) {
                fin_code[v] = pc;
                continue;
            }
            get_list(pool, pc, ids);
            for (uint32_t f = nodes[v].fin_lo; f < nodes[v].fin_hi; f++)
                ids.insert(std::upper_bound(ids.begin(), ids.end(), order[f]), order[f]);
            if (put_list(pool, ids, &fin_code[v]))
                return set_error(PFAC_ENOMEM, "pfac_build: output lists exceed %u words",
                                 FIN_MAX_OFF);
            n_lists++;
        }
        if (pool.empty()) pool.push_back(0);

        // ---- reduction step 2 (Section 3.2): equal subtrees of the last three
        // levels merged.  A node whose subtree is at most three levels tall
        // (height 0 to 2) is a tail node; tail nodes with equal finality and
        // equal children (symbols and merged children, compared bottom up)
        // become one merged node, so the leaves become one (step 1, Eq. 2).  The other nodes (the root and every node of height >= 3)
        // stay tree nodes.  Merged nodes cannot hold path-dependent outputs:
        // a walk that stops below its last tree node u after d symbols finds
        // its output in a side table keyed by (u, d, those d symbols).
        const bool dag = (o.flags & PFAC_BUILD_SUFFIX_MERGE) != 0;
        std::vector<uint8_t> upper;      // per tree node: kept as a tree node
        std::vector<uint32_t> canon;     // per tail node: its merged node
        std::vector<uint32_t> canon_rep; // per merged node: a tree node it stands for
        if (dag) {
            std::vector<uint32_t> h(Q, 0);
            for (uint64_t v = Q; v-- > 0;) {  // breadth-first: children after parents
                uint32_t m = 0;
                for (uint32_t c = 0; c < nodes[v].n_child; c++)
                    m = std::max(m, h[nodes[v].first_child + c] + 1);
                h[v] = m;
            }
            upper.assign(Q, 0);
            canon.assign(Q, 0xFFFFFFFFu);
            for (uint64_t v = 0; v < Q; v++) upper[v] = v == 0 || h[v] >= 3;
            std::unordered_map<std::string, uint32_t> sig;
            std::string key;
            for (uint32_t hh = 0; hh < 3; hh++)
                for (uint64_t v = 1; v < Q; v++) {
                    if (h[v] != hh) continue;
                    key.clear();
                    key.push_back(nodes[v].fin_lo != nodes[v].fin_hi ? 1 : 0);
                    const uint32_t *b = &bm[(uint64_t)v * W];
                    uint32_t ci = nodes[v].first_child;
                    for (uint32_t w = 0; w < W; w++)
                        for (uint32_t m = b[w]; m; m &= m - 1) {
                            const uint32_t c = 32 * w + (uint32_t)__builtin_ctz(m);
                            const uint32_t cc = canon[ci++];
                            key.push_back((char)c);
                            key.append(reinterpret_cast<const char *>(&cc), 4);
                        }
                    auto it = sig.find(key);
                    if (it != sig.end()) {
                        canon[v] = it->second;
                    } else {
                        canon[v] = (uint32_t)canon_rep.size();
                        sig.emplace(key, canon[v]);
                        canon_rep.push_back((uint32_t)v);
                    }
                }
        }

        // ---- leaf merge (Eq. 2) and record numbering ----------------------
        // (the dense layout numbers every node the same way, without merges)
        const bool dense = o.layout == PFAC_LAYOUT_DENSE;
        std::vector<uint8_t> all_leaf(Q, 0);
        uint64_t n_leaves = 0;
        for (uint64_t v = 0; v < Q; v++) {
            if (v > 0 && nodes[v].n_child == 0) n_leaves++;
            if (nodes[v].n_child && !dag && !dense) {
                bool all = true;
                for (uint32_t c = 0; c < nodes[v].n_child && all; c++)
                    all = nodes[nodes[v].first_child + c].n_child == 0;
                all_leaf[v] = all;
            }
        }
        // Record order: sibling groups are placed breadth-first, each group
        // contiguous and in symbol order (what Eq. 1 needs); below a group,
        // every single-child chain continues in consecutive records, so a
        // walk along a chain can fetch several levels in one memory round.
        const uint32_t NOREC = 0xFFFFFFFFu;
        std::vector<uint32_t> rec_of(Q, NOREC);
        uint32_t n_rec = 0;
        uint64_t merged = 0;
        for (uint64_t v = 1; v < Q && !dag; v++)
            if (nodes[v].n_child == 0 && all_leaf[nodes[v].parent]) merged++;
        // With the merge, only tree nodes are placed this way (a tail node's
        // record is its merged node's, after all tree records); the tree
        // children of a node whose children are all tree nodes stay one
        // contiguous group.
        auto rec_children = [&](uint32_t v) -> uint32_t {
            if (dag) return upper[v] ? nodes[v].n_child : 0u;
            return all_leaf[v] ? 0u : nodes[v].n_child;
        };
        auto placed = [&](uint32_t c) { return !dag || upper[c]; };
        std::vector<uint32_t> groups;  // nodes whose child group is still to place
        groups.reserve(Q / 2 + 1);
        auto place_chain = [&](uint32_t m) {
            while (rec_children(m) == 1 && placed(nodes[m].first_child)) {
                m = nodes[m].first_child;
                rec_of[m] = n_rec++;
            }
            if (rec_children(m) >= 1) groups.push_back(m);
        };
        uint32_t n_upper = 0;
        rec_of[0] = n_rec++;
        place_chain(0);
        for (size_t gi = 0; gi < groups.size(); gi++) {
            const uint32_t v = groups[gi];
            const uint32_t f = nodes[v].first_child, nc = nodes[v].n_child;
            for (uint32_t c = 0; c < nc; c++)
                if (placed(f + c)) rec_of[f + c] = n_rec++;
            for (uint32_t c = 0; c < nc; c++)
                if (placed(f + c)) place_chain(f + c);
        }
        if (dag) {
            n_upper = n_rec;
            if ((uint64_t)n_upper + canon_rep.size() >= (1ull << D_TAIL_SHIFT))
                return set_error(PFAC_EINVAL, "pfac_build: merged trie too large");
            for (uint64_t v = 1; v < Q; v++)
                if (!upper[v]) rec_of[v] = n_upper + canon[v];
            n_rec = n_upper + (uint32_t)canon_rep.size();
        }

        // ---- prefix nodes -------------------------------------------------
        // depths kmin..kdef: the default depth keeps the bitmap F_k at most
        // 2^20 bits (128 KiB), small enough for shared memory
        const uint32_t bps = bits_per_symbol(sigma);
        const uint32_t klim = std::min<uint32_t>(std::max(1u, 20 / bps), KMAX);
        // every prefix index spans at least 5 bits, so that its low 5 bits
        // address a bit within a 32-bit bitmap word
        const uint32_t kfloor = (5 + bps - 1) / bps;
        if (o.prefix_depth > klim)
            return set_error(PFAC_EINVAL, "pfac_build: prefix_depth %u > %u", o.prefix_depth, klim);
        if (o.prefix_depth && o.prefix_depth < kfloor)
            return set_error(PFAC_EINVAL, "pfac_build: prefix_depth %u < %u for this alphabet",
                             o.prefix_depth, kfloor);
        // record format: one packed word per node for alphabets of up to 8
        // symbols when every base fits below the bitmap (bases index records,
        // merged-leaf outputs or the indirection list, each fewer than Q)
        const uint32_t psh = pk_shift(sigma);
        const bool packed = !dense && sigma <= 8 && !(o.flags & PFAC_BUILD_WIDE_RECORDS) &&
                            Q < (1ull << psh);
        const uint32_t F = packed ? 0u : W;
        // the merged trie's kernel instances take each alphabet's own format
        if (dag && sigma <= 8 && !packed)
            return set_error(PFAC_EINVAL, "pfac_build: the suffix merge takes packed records for "
                             "alphabets of up to 8 symbols (no PFAC_BUILD_WIDE_RECORDS; fewer than "
                             "2^%u nodes)", psh);
        const int RW = rec_words((int)F);
        // entries of the prefix node of each depth: the indices whose walk
        // reaches depth k, plus those that stop earlier after a final (a
        // node of depth d < k with output, on a symbol value it has no child
        // on, any symbols after)
        uint64_t n_ent[KMAX + 1] = {0};
        for (uint64_t v = 0; v < Q; v++) {
            const uint32_t d = nodes[v].depth;
            if (d > klim) continue;
            const uint64_t miss = (1ull << bps) - nodes[v].n_child;
            for (uint32_t k = std::max(d, kfloor); k <= klim; k++) {
                if (k == d) n_ent[k] += 1;
                else if (fin_code[v]) n_ent[k] += miss << ((k - d - 1) * bps);
            }
        }
        // Default depth: the shallowest that passes at most 1/256 of uniform
        // windows, among the depths whose entries stay within a quarter of
        // the records' bytes (64 KiB at least); the deepest of those when
        // none is that selective.
        uint32_t kdef = o.prefix_depth;
        if (!kdef) {
            // (the dense layout takes the depth its compressed table would)
            const int rw_c = (sigma <= 8 && Q < (1ull << psh)) ? 1 : rec_words((int)W);
            const uint64_t budget = std::max<uint64_t>(64 * 1024, (uint64_t)n_rec * rw_c);
            uint32_t kcap = kfloor;
            for (uint32_t k = kfloor; k <= klim; k++)
                if (n_ent[k] * 4 <= budget) kcap = k;
            kdef = kcap;
            for (uint32_t k = kfloor; k <= kcap; k++)
                if (n_ent[k] * 256 <= (1ull << (k * bps))) {
                    kdef = k;
                    break;
                }
        }
        const uint32_t kmin = std::max(kdef > 2 ? kdef - 2 : 1u, kfloor);
        const uint32_t kmax = kdef;
        // walk the node-level trie over k symbols packed in x
        auto child_of = [&](uint32_t v, uint32_t c) -> int64_t {
            if (c >= sigma) return -1;
            const uint32_t *b = &bm[(uint64_t)v * W];
            if (!((b[c >> 5] >> (c & 31)) & 1)) return -1;
            uint32_t r = 0;
            for (uint32_t w = 0; w < (c >> 5); w++) r += __builtin_popcount(b[w]);
            r += __builtin_popcount(b[c >> 5] & ((1u << (c & 31)) - 1));
            return (int64_t)nodes[v].first_child + r;
        };

        // ---- section sizes ------------------------------------------------
        uint64_t sz_rec = dense ? 0 : (uint64_t)n_rec * RW * 4;
        uint64_t sz_fin = (!dense && F == 1) ? (uint64_t)n_rec * 4 : 0;
        std::vector<uint32_t> leaf_fin;
        if (!dense) {
            leaf_fin.reserve(merged);
        }
        uint64_t sz_pool = pool.size() * 4;
        // prefix node of depth k: bitmap, block counts, entries (Eq. 1 on the
        // collapsed first k levels)
        std::vector<uint32_t> Fv[KMAX + 1], Cv[KMAX + 1], Ev[KMAX + 1], Mv[KMAX + 1];
        std::vector<uint8_t> Bv[KMAX + 1];
        uint32_t cshift[KMAX + 1] = {0};
        uint64_t sz_F[KMAX + 1] = {0}, sz_C[KMAX + 1] = {0}, sz_E[KMAX + 1] = {0},
                 sz_M[KMAX + 1] = {0}, sz_B[KMAX + 1] = {0};
        for (uint32_t k = kmin; k <= kmax; k++) {
            const uint64_t ent = 1ull << (k * bps);
            const uint32_t smask = (1u << bps) - 1;
            const uint64_t fw = ent >= 32 ? ent / 32 : 1;
            // a count per word keeps the rank to one count and one popcount;
            // large bitmaps count per 8 words
            const uint32_t cs = fw <= 8192 ? 0u : 3u;
            Fv[k].assign(fw, 0);
            Cv[k].assign((fw + (1ull << cs) - 1) >> cs, 0);
            cshift[k] = cs;
            // prefix bytes where the planner would use them (the bitmap
            // passes at least 1% of windows)
            const bool with_b = k * bps <= BYTES_MAX_BITS && n_ent[k] * 100 >= ent;
            if (with_b) Bv[k].assign(ent < 4 ? 4 : ent, 0);
            for (uint64_t x = 0; x < ent; x++) {
                uint32_t v = 0, e = 0;
                bool stopped = false;
                for (uint32_t i = 0; i < k; i++) {
                    const int64_t ch = child_of(v, (uint32_t)(x >> (bps * i)) & smask);
                    if (ch < 0) {
                        e = fin_code[v];
                        stopped = true;
                        break;
                    }
                    v = (uint32_t)ch;
                }
                uint32_t mask = 0xFFFFFFFFu, bucket = 0xFFu;
                if (!stopped) {
                    if (nodes[v].n_child == 0) {
                        e = fin_code[v];  // a leaf ends the walk
                    } else {
                        e = D_CONT | rec_of[v];
                        if (dag && !upper[v]) {
                            // a tail record: the entry names the last tree
                            // record and the depth below it instead
                            uint32_t u = v, d = 0;
                            while (!upper[u]) {
                                u = nodes[u].parent;
                                d++;
                            }
                            e = D_CONT | D_TAIL | (d << D_TAIL_SHIFT) | rec_of[u];
                        }
                        if (fin_code[v] == 0) {
                            mask = 0;
                            bucket = 0;
                            for (uint32_t c = 0; c < sigma; c++)
                                if ((bm[(uint64_t)v * W + (c >> 5)] >> (c & 31)) & 1) {
                                    mask |= 1u << child_hash(c, sigma);
                                    bucket |= 1u << byte_bucket(c, sigma);
                                }
                        }
                    }
                }
                if (e) {
                    Fv[k][x >> 5] |= 1u << (x & 31);
                    Ev[k].push_back(e);
                    Mv[k].push_back(mask);
                    if (with_b) Bv[k][x] = (uint8_t)bucket;
                }
            }
            uint32_t run = 0;
            for (uint64_t w = 0; w < fw; w++) {
                if ((w & ((1u << cs) - 1)) == 0) Cv[k][w >> cs] = run;
                run += __builtin_popcount(Fv[k][w]);
            }
            if (Ev[k].empty()) {
                Ev[k].push_back(0);
                Mv[k].push_back(0);
            }
            sz_F[k] = fw * 4;
            sz_C[k] = Cv[k].size() * 4;
            sz_E[k] = Ev[k].size() * 4;
            // narrow masks for small alphabets: mask_bits(sigma) bits per
            // entry, packed low entry first (an all-ones mask still means
            // "keep whatever follows")
            const uint32_t mb = mask_bits(sigma);
            if (mb < 32) {
                std::vector<uint32_t> packed((Mv[k].size() * mb + 31) / 32, 0);
                const uint32_t ones = (1u << mb) - 1u;
                for (size_t r = 0; r < Mv[k].size(); r++)
                    packed[(r * mb) >> 5] |= (Mv[k][r] & ones) << ((r * mb) & 31);
                Mv[k].swap(packed);
            }
            // child masks are only used from shared memory: none when the
            // entries could never fit there
            if (Mv[k].size() * 4 > MASKS_MAX_BYTES) Mv[k].clear();
            sz_M[k] = Mv[k].size() * 4;
            sz_B[k] = Bv[k].size();
        }
        // ---- gram filter over g = kmax + 1 symbols (see table.h) -----------
        uint32_t g_len = 0, g_bits = 0;
        uint64_t g_set = 0;
        std::vector<uint32_t> Gv;
        if ((kmax + 1) * bps <= 32) {
            g_len = kmax + 1;
            const uint32_t A = 1u << bps;  // packed symbol values (>= sigma: no child)
            // pass 0 counts the strings, pass 1 sets their bits
            for (int pass = 0; pass < 2; pass++) {
                // every string x + (any symbols at depths d .. g-1)
                auto add_all = [&](uint32_t x, uint32_t d) {
                    const uint64_t n = 1ull << (bps * (g_len - d));
                    if (pass == 0) {
                        g_set += n;
                        return;
                    }
                    const uint32_t gm = gram_mul(bps * g_len);
                    for (uint64_t y = 0; y < n; y++) {
                        const uint32_t s = x | (uint32_t)(y << (bps * d));
                        Gv[gram_word(s * gm, g_bits)] |= 1u << (s & 31);
                    }
                };
                std::vector<std::pair<uint32_t, uint32_t>> stack;  // node, packed prefix
                stack.push_back({0u, 0u});
                while (!stack.empty()) {
                    const uint32_t v = stack.back().first, x = stack.back().second;
                    stack.pop_back();
                    const uint32_t d = nodes[v].depth;
                    const uint32_t *b = &bm[(uint64_t)v * W];
                    uint32_t ci = nodes[v].first_child;
                    if (fin_code[v]) {
                        // v reports output: a missing child ends the walk with it
                        for (uint32_t c = 0; c < A; c++) {
                            const uint32_t xc = x | (c << (bps * d));
                            if (c < sigma && ((b[c >> 5] >> (c & 31)) & 1)) {
                                if (d + 1 == g_len) add_all(xc, g_len);
                                else stack.push_back({ci, xc});
                                ci++;
                            } else {
                                add_all(xc, d + 1);
                            }
                        }
                    } else {
                        for (uint32_t w = 0; w < W; w++)
                            for (uint32_t m = b[w]; m; m &= m - 1) {
                                const uint32_t c = 32 * w + (uint32_t)__builtin_ctz(m);
                                const uint32_t xc = x | (c << (bps * d));
                                if (d + 1 == g_len) add_all(xc, g_len);
                                else stack.push_back({ci, xc});
                                ci++;
                            }
                    }
                }
                if (pass == 0 && g_set > (1ull << 26)) {
                    // too many strings for a useful filter: none
                    g_len = 0;
                    g_set = 0;
                    break;
                }
                if (pass == 0) {
                    // about 64 bits per string, within [2^10, 2^20] bits (the
                    // planner folds it down to fit shared memory)
                    g_bits = GRAM_MIN_BITS;
                    while (g_bits < GRAM_MAX_BITS && (1ull << g_bits) < 64 * g_set) g_bits++;
                    // larger pattern sets get room for a sparse first stage even
                    // when few strings are set (the planner folds it as needed)
                    const uint32_t floor_bits = n_patterns >= 1000 ? 20u : (n_patterns >= 100 ? 18u : 0u);
                    if (g_bits < floor_bits) g_bits = floor_bits;
                    Gv.assign((1ull << g_bits) / 32, 0);
                }
            }
        }
        const uint64_t sz_G = Gv.size() * 4;
        // truncated tables keep the patterns for verification
        std::vector<uint32_t> pat_off;
        std::vector<uint8_t> pat_bytes;
        if (o.truncate_depth) {
            pat_off.resize((size_t)n_patterns + 1, 0);
            for (uint32_t i = 0; i < n_patterns; i++) pat_off[i + 1] = pat_off[i] + pats[i].len;
            pat_bytes.resize(std::max<uint64_t>(pat_off[n_patterns], 4));
            for (uint32_t i = 0; i < n_patterns; i++)
                memcpy(pat_bytes.data() + pat_off[i], pats[i].p, pats[i].len);
        }
        const uint64_t sz_po = pat_off.size() * 4, sz_pb = pat_bytes.size();

        uint64_t sz_stt = dense ? Q * sigma * 4 : 0;
        uint64_t sz_dfin = dense ? Q * 4 : 0;

        // records and merged-leaf outputs
        std::vector<uint32_t> rec, finv, ind;
        if (!dense) {
            rec.assign((uint64_t)n_rec * RW, 0);
            if (F <= 1) finv.assign(n_rec, 0);
            for (uint64_t v = 0; v < Q; v++) {
                uint32_t r = rec_of[v];
                if (r == NOREC) continue;
                // a merged node's record comes from the one tree node it keeps
                if (dag && !upper[v] && canon_rep[canon[v]] != v) continue;
                uint32_t *R = &rec[(uint64_t)r * RW];
                uint32_t meta = 0;
                if (dag && nodes[v].n_child) {
                    // children through the indirection list unless they are all
                    // tree nodes (then consecutive records, Eq. 1 directly)
                    bool direct = upper[v] != 0;
                    for (uint32_t c = 0; c < nodes[v].n_child && direct; c++)
                        direct = upper[nodes[v].first_child + c] != 0;
                    if (direct) {
                        meta = rec_of[nodes[v].first_child];
                        for (uint32_t c = 0; c < nodes[v].n_child; c++)
                            if (rec_of[nodes[v].first_child + c] != meta + c)
                                return set_error(PFAC_EDEVICE, "pfac_build: internal error (dag)");
                    } else {
                        // META_ALL_LEAF marks the record for the walk's slow
                        // path, which follows ind[] and tracks the tail
                        meta = META_ALL_LEAF | META_IND | (uint32_t)ind.size();
                        for (uint32_t c = 0; c < nodes[v].n_child; c++)
                            ind.push_back(rec_of[nodes[v].first_child + c]);
                    }
                } else if (all_leaf[v]) {
                    meta = META_ALL_LEAF | (uint32_t)leaf_fin.size();
                    for (uint32_t c = 0; c < nodes[v].n_child; c++)
                        leaf_fin.push_back(fin_code[nodes[v].first_child + c]);
                } else if (nodes[v].n_child) {
                    meta = rec_of[nodes[v].first_child];
                    // children of a node with an internal child all keep records,
                    // contiguous in breadth-first order
                    for (uint32_t c = 0; c < nodes[v].n_child; c++)
                        if (rec_of[nodes[v].first_child + c] != meta + c)
                            return set_error(PFAC_EDEVICE, "pfac_build: internal error (records)");
                }
                // a merged node's outputs depend on the path: the side table
                const uint32_t fv = dag && !upper[v] ? 0u : fin_code[v];
                if (F == 0) {
                    // on a merged trie the flag marks the records with
                    // indirect children (leaf merge is off there)
                    R[0] = (meta & META_ALL_LEAF) | (fv ? PK_FIN : 0u) | (bm[v * W] << psh) |
                           (meta & META_BASE_MASK);
                    finv[r] = fv;
                    continue;
                }
                for (uint32_t w = 0; w < W; w++) R[w] = bm[v * W + w];
                if (W == 1) {
                    R[1] = meta;
                    finv[r] = fv;
                } else if (W == 2) {
                    R[2] = meta;
                    R[3] = fv;
                } else {
                    R[8] = meta;
                    R[9] = fv;
                    uint32_t cum = 0;
                    uint32_t c4[2] = {0, 0};
                    for (uint32_t w = 0; w < 8; w++) {
                        c4[w >> 2] |= cum << (8 * (w & 3));
                        cum += __builtin_popcount(bm[v * W + w]);
                    }
                    R[10] = c4[0];
                    R[11] = c4[1];
                }
            }
        }
        if (leaf_fin.empty()) leaf_fin.push_back(0);
        uint64_t sz_leaf = dense ? 0 : leaf_fin.size() * 4;
        // packed records: outputs of the records that have one, by rank
        std::vector<uint32_t> fbc, fvals;
        if (F == 0) {
            const uint64_t nw = (uint64_t)n_rec / 32 + 1;
            fbc.assign(2 * nw, 0);
            uint32_t cnt = 0;
            for (uint64_t w = 0; w < nw; w++) {
                fbc[2 * w + 1] = cnt;
                for (uint32_t b = 0; b < 32; b++) {
                    const uint64_t r = 32 * w + b;
                    if (r < n_rec && finv[r]) {
                        fbc[2 * w] |= 1u << b;
                        fvals.push_back(finv[r]);
                        cnt++;
                    }
                }
            }
            if (fvals.empty()) fvals.push_back(0);
        }
        const uint64_t sz_fbc = fbc.size() * 4, sz_fv = F == 0 ? fvals.size() * 4 : 0;
        if (ind.empty()) ind.push_back(0);
        const uint64_t sz_ind = dag ? ind.size() * 4 : 0;

        // side table of the merged trie: for every tail node with output, the
        // output under the key (its last tree ancestor's record, the depth
        // below it, the symbols from there); open addressing, linear probes
        std::vector<uint64_t> side_keys;
        std::vector<uint32_t> side_vals;
        uint32_t side_slots = 0;
        uint64_t side_n = 0;
        if (dag) {
            std::vector<uint64_t> ks;
            std::vector<uint32_t> vs;
            for (uint64_t v = 1; v < Q; v++) {
                if (upper[v] || !fin_code[v]) continue;
                uint32_t u = (uint32_t)v, tp = 0, d = 0;
                uint32_t syms[4] = {0, 0, 0, 0};
                while (!upper[u]) {
                    syms[d++] = sym_at(nodes[u].lo, nodes[u].depth - 1);
                    u = nodes[u].parent;
                }
                for (uint32_t i = 0; i < d; i++) tp |= syms[d - 1 - i] << (bps * i);
                ks.push_back(dag_side_key(rec_of[u], d, tp));
                vs.push_back(fin_code[v]);
            }
            side_n = ks.size();
            side_slots = (uint32_t)std::max<uint64_t>(16, side_n + side_n / 4 + 1);
            side_keys.assign(side_slots, DAG_SIDE_EMPTY);
            side_vals.assign(side_slots, 0);
            for (size_t i = 0; i < ks.size(); i++) {
                uint64_t h = dag_side_slot(ks[i], side_slots);
                while (side_keys[h] != DAG_SIDE_EMPTY) h = h + 1 == side_slots ? 0 : h + 1;
                side_keys[h] = ks[i];
                side_vals[h] = vs[i];
            }
        }
        const uint64_t sz_sk = side_keys.size() * 8, sz_sv = side_vals.size() * 4;

        // blob layout
        uint64_t off = 0;
        auto place = [&](uint64_t sz) {
            uint64_t at = off;
            off = align16(off + sz);
            return at;
        };
        uint64_t o_rec = place(sz_rec), o_fin = place(sz_fin), o_leaf = place(sz_leaf),
                 o_pool = place(sz_pool), o_fbc = place(sz_fbc), o_fv = place(sz_fv);
        const uint64_t o_ind = place(sz_ind), o_sk = place(sz_sk), o_sv = place(sz_sv);
        uint64_t o_F[KMAX + 1] = {0}, o_C[KMAX + 1] = {0}, o_E[KMAX + 1] = {0},
                 o_M[KMAX + 1] = {0}, o_B[KMAX + 1] = {0};
        for (uint32_t k = kmin; k <= kmax; k++) {
            o_F[k] = place(sz_F[k]);
            o_C[k] = place(sz_C[k]);
            o_E[k] = place(sz_E[k]);
            o_M[k] = place(sz_M[k]);
            o_B[k] = place(sz_B[k]);
        }
        const uint64_t o_G = place(sz_G);
        const uint64_t o_po = place(sz_po), o_pb = place(sz_pb);
        uint64_t o_stt = place(sz_stt), o_dfin = place(sz_dfin);
        const uint64_t blob = std::max<uint64_t>(off, 256);

        std::vector<uint8_t> host;
        host.assign(blob, 0);
        auto put = [&](uint64_t at, const void *src, uint64_t n) {
            if (n) memcpy(host.data() + at, src, n);
        };
        put(o_rec, rec.data(), sz_rec);
        put(o_fin, finv.data(), sz_fin);
        put(o_fbc, fbc.data(), sz_fbc);
        put(o_fv, fvals.data(), sz_fv);
        put(o_leaf, leaf_fin.data(), sz_leaf);
        put(o_pool, pool.data(), sz_pool);
        put(o_ind, ind.data(), sz_ind);
        put(o_sk, side_keys.data(), sz_sk);
        put(o_sv, side_vals.data(), sz_sv);
        for (uint32_t k = kmin; k <= kmax; k++) {
            put(o_F[k], Fv[k].data(), sz_F[k]);
            put(o_C[k], Cv[k].data(), sz_C[k]);
            put(o_E[k], Ev[k].data(), sz_E[k]);
            put(o_M[k], Mv[k].data(), sz_M[k]);
            put(o_B[k], Bv[k].data(), sz_B[k]);
        }
        put(o_G, Gv.data(), sz_G);
        put(o_po, pat_off.data(), sz_po);
        put(o_pb, pat_bytes.data(), sz_pb);
        if (dense) {
            uint32_t *S = (uint32_t *)(host.data() + o_stt);
            uint32_t *DF = (uint32_t *)(host.data() + o_dfin);
            // state numbers are the record numbers (chains consecutive); the
            // root is 0 and never a child, so 0 marks "no child"
            for (uint64_t v = 0; v < Q; v++) {
                const uint64_t sv = rec_of[v];
                DF[sv] = fin_code[v];
                uint32_t r = 0;
                for (uint32_t c = 0; c < sigma; c++)
                    if ((bm[v * W + (c >> 5)] >> (c & 31)) & 1)
                        S[sv * sigma + c] = rec_of[nodes[v].first_child + r++];
            }
        }

        // ---- upload -------------------------------------------------------
        pfac_table *t = new (std::nothrow) pfac_table();
        if (!t) return set_error(PFAC_ENOMEM, "pfac_build: host allocation failed");
        const bool host_only = (o.flags & PFAC_BUILD_HOST_ONLY) != 0;
        cudaStream_t st = (cudaStream_t)cuda_stream;
        cudaError_t ce = cudaSuccess;
        if (!host_only) {
            cudaGetDevice(&t->device);
            ce = cudaMalloc(&t->d_blob, blob);
            if (ce != cudaSuccess) {
                delete t;
                cudaGetLastError();
                return set_error(ce == cudaErrorMemoryAllocation ? PFAC_ENOMEM : PFAC_ECUDA,
                                 "pfac_build: cudaMalloc(%llu): %s", (unsigned long long)blob,
                                 cudaGetErrorString(ce));
            }
            ce = cudaMemcpyAsync(t->d_blob, host.data(), blob, cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
            if (ce != cudaSuccess) {
                cudaFree(t->d_blob);
                delete t;
                return set_error(PFAC_ECUDA, "pfac_build: upload: %s", cudaGetErrorString(ce));
            }
        }
        t->blob_bytes = blob;
        if (host_only) t->h_blob = std::move(host);
        uint8_t *B = host_only ? t->h_blob.data() : (uint8_t *)t->d_blob;
        DevTable &dv = t->dev;
        memset(&dv, 0, sizeof(dv));
        dv.sigma = sigma;
        dv.W = dense ? 3u : F;  // 3: rows of the dense transition table
        dv.pk_shift = psh;
        dv.bps = bps;
        dv.kdef = kdef;
        dv.kmin = kmin;
        dv.layout = o.layout;
        dv.max_len = max_len;
        dv.n_rec = n_rec;
        dv.n_nodes = (uint32_t)Q;
        dv.rec = (const uint32_t *)(B + (dense ? o_stt : o_rec));
        dv.fin = (const uint32_t *)(B + o_fin);
        dv.fbc = F == 0 ? (const uint32_t *)(B + o_fbc) : nullptr;
        dv.fvals = F == 0 ? (const uint32_t *)(B + o_fv) : nullptr;
        dv.n_fvals = F == 0 ? (uint32_t)fvals.size() : 0u;
        dv.leaf_fin = (const uint32_t *)(B + o_leaf);
        dv.pool = (const uint32_t *)(B + o_pool);
        dv.pool_words = (uint32_t)pool.size();
        dv.leaf_words = (uint32_t)leaf_fin.size();
        dv.dag = dag ? 1u : 0u;
        dv.n_upper = dag ? n_upper : n_rec;
        dv.ind = (const uint32_t *)(B + o_ind);
        dv.ind_words = dag ? (uint32_t)ind.size() : 0u;
        dv.side_keys = dag ? (const uint64_t *)(B + o_sk) : nullptr;
        dv.side_vals = dag ? (const uint32_t *)(B + o_sv) : nullptr;
        dv.side_slots = side_slots;
        for (uint32_t k = kmin; k <= kmax; k++) {
            dv.F[k] = (const uint32_t *)(B + o_F[k]);
            dv.C[k] = (const uint32_t *)(B + o_C[k]);
            dv.E[k] = (const uint32_t *)(B + o_E[k]);
            dv.M[k] = sz_M[k] ? (const uint32_t *)(B + o_M[k]) : nullptr;
            dv.c_shift[k] = cshift[k];
            dv.n_e[k] = (uint32_t)Ev[k].size();
            dv.m_words[k] = (uint32_t)Mv[k].size();
            dv.B[k] = sz_B[k] ? (const uint8_t *)(B + o_B[k]) : nullptr;
        }
        dv.G = g_len ? (const uint32_t *)(B + o_G) : nullptr;
        dv.trunc = o.truncate_depth;
        dv.n_pat = n_patterns;
        dv.pat_off = sz_po ? (const uint32_t *)(B + o_po) : nullptr;
        dv.pat = sz_pb ? (const uint8_t *)(B + o_pb) : nullptr;
        dv.g_len = g_len;
        dv.g_bits = g_bits;
        dv.g_set = g_set;
        dv.stt = dense ? (const uint32_t *)(B + o_stt) : nullptr;
        dv.dfin = dense ? (const uint32_t *)(B + o_dfin) : nullptr;
        t->kmax = kmax;
        t->kmin = kmin;

        t->match_density = match_density;
        pfac_table_info_t &I = t->info;
        I.alphabet_size = sigma;
        I.n_patterns = n_patterns;
        I.min_len = min_len;
        I.max_len = max_len;
        I.layout = o.layout;
        I.prefix_depth = dv.kdef;
        I.trie_nodes = Q;
        I.trie_leaves = n_leaves;
        I.records = dense ? Q : n_rec;
        I.merged_leaves = dense ? 0 : merged;
        I.device_bytes = blob;
        I.paper_bytes = Q * ((sigma + 7) / 8 + 4);
        I.dense_bytes = Q * 4ull * sigma;
        I.output_lists = n_lists;
        I.output_list_words = pool.size();
        I.gram_len = g_len;
        I.gram_bits = g_bits;
        I.gram_strings = g_set;
        I.merged_trie_nodes = dag ? (uint64_t)n_upper + canon_rep.size() : 0;
        I.side_entries = side_n;
        I.trie_bytes = sz_rec + sz_fin + sz_fbc + sz_fv + sz_leaf + sz_pool + sz_ind + sz_sk + sz_sv;
        I.index_bytes = sz_G;
        for (uint32_t k = kmin; k <= kmax; k++)
            I.index_bytes += sz_F[k] + sz_C[k] + sz_E[k] + sz_M[k] + sz_B[k];
        // the dense layout's transition table and outputs are its trie
        if (dense) I.trie_bytes += sz_stt + sz_dfin;
        I.other_bytes = sz_po + sz_pb;
        I.record_bytes = dense ? 0u : (uint32_t)RW * 4u;
        *out = t;
        return PFAC_OK;
    } catch (const std::bad_alloc &) {
        return set_error(PFAC_ENOMEM, "pfac_build: host allocation failed");
    }
}

extern "C" int pfac_table_info(const pfac_table *t, pfac_table_info_t *out) {
    if (!t || !out) return set_error(PFAC_EINVAL, "pfac_table_info: NULL argument");
    *out = t->info;
    return PFAC_OK;
}

extern "C" void pfac_table_free(pfac_table *t) {
    if (!t) return;
    if (t->d_blob) {
        int cur = 0;
        cudaGetDevice(&cur);
        if (cur != t->device) cudaSetDevice(t->device);
        cudaFree(t->d_blob);
        if (cur != t->device) cudaSetDevice(cur);
    }
    delete t;
}

extern "C" const char *pfac_status_str(int s) {
    switch (s) {
        case PFAC_OK: return "ok";
        case PFAC_EINVAL: return "invalid argument";
        case PFAC_EDUP: return "duplicate pattern";
        case PFAC_ESYMBOL: return "pattern symbol outside the alphabet";
        case PFAC_ENOMEM: return "out of memory";
        case PFAC_ENOSPC: return "output capacity too small";
        case PFAC_ECUDA: return "CUDA error";
        case PFAC_ETIMEOUT: return "device wait timed out";
        case PFAC_EDEVICE: return "device consistency check failed";
        case PFAC_EIO: return "table file I/O failed";
        case PFAC_EFORMAT: return "not a table file of this format";
        default: return "unknown status";
    }
}

extern "C" int pfac_last_error(char *buf, size_t n) {
    if (buf && n) {
        strncpy(buf, g_last_msg, n - 1);
        buf[n - 1] = 0;
    }
    return g_last_status;
}

extern "C" int pfac_version(void) { return 200; }

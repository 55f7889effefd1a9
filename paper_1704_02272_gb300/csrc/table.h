// Device-side view of a matching table and the encodings shared by the host
// builder (builder.cpp) and the kernels (match.cu).
//
// Compressed layout (Sections 3.1 and 3.2):
//   * Trie nodes are numbered breadth-first over the alphabetically sorted
//     patterns; siblings are contiguous and in symbol order (Section 3.1).
//   * A node record holds a bitmap of W = ceil(sigma/32) words (bit c set when
//     the node has a child on symbol c) and a base; the child on c is
//     base + rank(c), rank(c) = number of bitmap bits below c (Eq. 1).
//   * Leaf merge (Eq. 2): leaves have no children, so a node whose children
//     are all leaves keeps no records for them; its base then indexes
//     leaf_fin[], which holds each merged leaf's output list, and its meta word
//     carries META_ALL_LEAF.  Leaves with an internal sibling keep a record
//     with an empty bitmap.
//   * Output: every state s carries fin(s), the sorted ids of all patterns
//     that are prefixes of s's string (its final ancestors and itself).  A
//     walk reports fin of the state where it stops, which is exactly the set
//     of finals it passed (Section 2.3).
//   * Prefix node: the first k trie levels collapse into one node of fan-out
//     2^(k*BPS) (k symbols packed BPS bits each, first symbol lowest).  Its
//     bitmap F_k marks the indices whose walk does something (reaches depth k
//     or stops after a final); like a node record, its children are addressed
//     by popcount rank (Eq. 1): C_k holds the count of set bits before each
//     word (small bitmaps) or each 8 words, and E_k the entries of the set
//     bits in index order.  An
//     entry is D_CONT | record of the depth-k state, or the fin of the state
//     where a shorter walk stopped.  M_k holds per entry a 32-bit mask of the
//     hashed symbols (child_hash) the depth-k state has children on, or all
//     ones when the entry itself reports output: a survivor whose next symbol
//     misses the mask stops silently without visiting the records.
//
// Gram filter (an optional first on-chip stage): a bitmap G of 2^hb bits
// over strings of g symbols (packed like a prefix index).  Bit gram_pos(x)
// is set for every string x whose walk from the root reaches depth g, or
// stops before depth g at a state that reports output; a start position
// whose next g symbols miss G reports nothing.  Hashing keeps G small when
// 2^(g*b) is far beyond shared memory; collisions only let extra positions
// through to the exact prefix-node test.
//
// Merged trie (reduction step 2 of Section 3.2, build flag
// PFAC_BUILD_SUFFIX_MERGE): equal subtrees of at most three levels share one
// record each (tail records, numbered from n_upper on).  A record whose
// children are not all consecutive tree records carries META_IND: child c is
// ind[base + rank(c)].  Tail records hold no output; a walk that stops
// below its last tree record u after d symbols s_0 .. s_{d-1} finds its
// output (the fin of the tree node it reached) in the side table under
// dag_side_key(u, d, s_0 | s_1 << bps | ...), absent meaning none.  A
// prefix entry whose depth-k state is a tail record names u and d instead
// (D_TAIL).
//
// Dense layout (uncompressed PFAC): stt[s * sigma + c] = child or 0 (the root
// is never a child), dfin[s] = fin(s).
#pragma once
#include <stdint.h>

namespace pfac {

constexpr int KMAX = 16;                 // largest prefix depth held
constexpr uint64_t MASKS_MAX_BYTES = 96 * 1024;  // child masks kept up to this size
constexpr uint32_t META_ALL_LEAF = 0x80000000u;
constexpr uint32_t META_IND = 0x40000000u;        // merged trie: children through ind[]
constexpr uint32_t META_BASE_MASK = 0x3FFFFFFFu;
constexpr uint32_t D_CONT = 0x80000000u;  // prefix entry: continue at record
constexpr uint32_t D_VAL_MASK = 0x7FFFFFFFu;
// merged trie: a prefix entry whose state is a tail record holds D_CONT |
// D_TAIL | d << D_TAIL_SHIFT | u (u the last tree record above the state, d
// its depth below u; merged tries keep fewer than 2^28 records)
constexpr uint32_t D_TAIL = 0x40000000u;
constexpr uint32_t D_TAIL_SHIFT = 28;
constexpr uint32_t D_TAIL_REC = (1u << D_TAIL_SHIFT) - 1u;
// fin encoding: 0 = empty; else (off << FIN_LEN_BITS) | len, len < FIN_LEN_ESC
// with ids at pool[off .. off+len); len == FIN_LEN_ESC means the length is
// pool[off] and the ids follow it.
constexpr int FIN_LEN_BITS = 6;
constexpr uint32_t FIN_LEN_ESC = (1u << FIN_LEN_BITS) - 1;
constexpr uint32_t FIN_MAX_OFF = (1u << (31 - FIN_LEN_BITS)) - 1;

// 32-bit words per record for W bitmap words
//   W == 0: one packed word for alphabets of up to 8 symbols: bit 31 the
//           all-leaf flag (on a merged trie: children through ind[]), bit 30
//           set when the record has an output (PK_FIN), the bitmap's SB bits
//           (SB = 4 for sigma <= 4, else 8) at bits PK_SHIFT .. 29
//           (PK_SHIFT = 30 - SB), the base below PK_SHIFT; the outputs of
//           the records with one in fvals[], found by rank:
//           fbc[r >> 5] = {bit r & 31 set when record r has an output, the
//           number of such records before the word}
//   W == 1: {bm, meta}                          (fin in a separate array)
//   W == 2: {bm0, bm1, meta, fin}
//   W == 8: {bm0..bm7, meta, fin, cum0..3, cum4..7} (cum: popcount of the
//           words before each word, one byte per word)
__host__ __device__ constexpr int rec_words(int W) {
    return W == 0 ? 1 : (W == 1 ? 2 : (W == 2 ? 4 : 12));
}
__host__ __device__ constexpr uint32_t pk_shift(uint32_t sigma) { return sigma <= 4 ? 26u : 22u; }
constexpr uint32_t PK_FIN = 0x40000000u;

// Side table of the merged trie: key of (tree record u, depth d below it,
// packed symbols tp), its slot (the key's Fibonacci hash scaled to the
// table's n slots, at most 80% of them taken; linear probing from there),
// the empty key.
constexpr uint64_t DAG_SIDE_EMPTY = ~0ull;
__host__ __device__ inline uint64_t dag_side_key(uint32_t u, uint32_t d, uint32_t tp) {
    return ((uint64_t)u << 32) | ((uint64_t)d << 28) | tp;
}
__host__ __device__ inline uint64_t dag_side_slot(uint64_t key, uint32_t n) {
    return (((key * 0x9E3779B97F4A7C15ull) >> 32) * (uint64_t)n) >> 32;
}

// Gram filter hash of a string x of n = g * bps <= 32 bits: y = x * m with
// m = GRAM_MUL << (32 - n) (Knuth's multiplicative hashing with the
// golden-ratio constant, on an n-bit word); the word is the top hb - 5 bits
// of y, the bit within the word the low 5 bits of x.  Because the low
// 32 - n bits of m are zero, y ignores the bits of x above n: a 32-bit
// window holding the string in its low bits hashes without a mask.
constexpr uint32_t GRAM_MUL = 0x9E3779B1u;
constexpr uint32_t GRAM_MIN_BITS = 10, GRAM_MAX_BITS = 20;
__host__ __device__ inline uint32_t gram_mul(uint32_t n) {
    return n >= 32 ? GRAM_MUL : GRAM_MUL << (32 - n);
}
__host__ __device__ inline uint32_t gram_word(uint32_t y, uint32_t hb) { return y >> (37 - hb); }

// Bits per child mask: 4 for alphabets of up to 4 symbols, 8 up to 8, else
// 32 (an all-ones mask: the entry reports output, or has every child).
__host__ __device__ inline uint32_t mask_bits(uint32_t sigma) {
    return sigma <= 4 ? 4u : (sigma <= 8 ? 8u : 32u);
}

// Prefix bytes (an optional first stage for prefix indices of at most 16
// bits): B_k[x] = 0 when index x has no entry; 0xFF when the entry reports
// output (or the state has children in every bucket); else bit byte_bucket(c)
// set for every child symbol c of the depth-k state.
constexpr uint32_t BYTES_MAX_BITS = 16;
__host__ __device__ inline uint32_t byte_bucket(uint32_t c, uint32_t sigma) {
    return sigma <= 8 ? c : ((c ^ (c >> 3) ^ (c >> 6)) & 7u);
}

// Bit of symbol c in a child mask: exact for alphabets of up to 32 symbols.
__host__ __device__ inline uint32_t child_hash(uint32_t c, uint32_t sigma) {
    return sigma <= 32 ? c : ((c ^ (c >> 5)) & 31u);
}

struct DevTable {
    uint32_t sigma;
    uint32_t W;           // record format: 0 (packed), 1, 2 or 8 (bitmap words)
    uint32_t pk_shift;    // W == 0: bit of the bitmap's symbol 0
    uint32_t bps;         // bits per symbol in prefix indices
    uint32_t kdef;        // default prefix depth
    uint32_t kmin;        // shallowest prefix depth held
    uint32_t layout;      // pfac_layout
    uint32_t max_len;
    uint32_t n_rec;
    uint32_t n_nodes;     // dense layout: states
    uint32_t pool_words;  // words of the output-list pool
    uint32_t leaf_words;  // words of leaf_fin
    const uint32_t *rec;
    const uint32_t *fin;      // W == 1 only
    const uint32_t *fbc;      // W == 0 only: {bits, count} word pairs per 32 records
    const uint32_t *fvals;    // W == 0 only: outputs of the records that have one
    uint32_t n_fvals;
    const uint32_t *leaf_fin;
    const uint32_t *pool;
    const uint32_t *F[KMAX + 1];   // prefix bitmap of depth k
    const uint32_t *C[KMAX + 1];   // set bits of F_k before each group of 2^c_shift words
    uint32_t c_shift[KMAX + 1];    // 0 (a count per word) or 3 (per 8 words)
    const uint32_t *E[KMAX + 1];   // entries of the set bits of F_k
    const uint32_t *M[KMAX + 1];   // per entry: hashed symbols its state continues with,
                                   // packed (nullptr when too large to be used)
    uint32_t n_e[KMAX + 1];        // number of entries of depth k
    uint32_t m_words[KMAX + 1];    // words of M_k (mask_bits(sigma) bits per entry)
    const uint8_t *B[KMAX + 1];    // prefix bytes of depth k (nullptr when k * bps > 16)
    const uint32_t *G;             // gram filter (nullptr when none)
    uint32_t g_len;                // g: symbols per gram
    uint32_t g_bits;               // hb: log2 of the bits of G
    uint64_t g_set;                // strings whose bit is set
    uint32_t trunc;           // truncation depth (0: exact table)
    const uint8_t *pat;       // truncated tables: the patterns' bytes,
    const uint32_t *pat_off;  //   pattern j at pat[pat_off[j] .. pat_off[j + 1])
    uint32_t n_pat;
    const uint32_t *stt;      // dense layout
    const uint32_t *dfin;
    // merged trie
    uint32_t dag;             // 1: records of the merged trie
    uint32_t n_upper;         // records below it are tree records (all, without the merge)
    const uint32_t *ind;      // child indirection
    uint32_t ind_words;
    uint32_t side_slots;      // slots of the side table
    const uint64_t *side_keys;
    const uint32_t *side_vals;
};

}  // namespace pfac

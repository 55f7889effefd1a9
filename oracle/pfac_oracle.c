/*
 * CPU oracle for exact multi-pattern matching.  TEST INFRASTRUCTURE ONLY:
 * only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * may load this code.  It shares nothing with the GPU path.
 *
 * What it computes (the problem statement of Section 2.2 with the start-
 * position semantics of the failure-less matcher of Section 2.3): given
 * distinct non-empty patterns P_0..P_{n-1}, a text T[0..N) and segment
 * offsets 0 = o_0 <= o_1 <= ... <= o_S = N, the set
 *
 *     M = { (p, j) : exists k with o_k <= p and p + |P_j| <= o_{k+1}
 *                    and T[p .. p+|P_j|) = P_j }
 *
 * sorted by p, then by j.  Two independent programs produce it:
 *
 *   O1 (obf_match)  brute force: every segment, every start p, every pattern
 *                   j, a length check then memcmp.  This is the definition
 *                   written out.
 *   O2 (oac_*)      the classic Aho-Corasick automaton with goto and failure
 *                   links (Section 2.2): one pass per segment, each match is
 *                   reported at its end position e and converted to the start
 *                   p = e - |P_j| + 1, then the list is sorted.
 *
 * Both take a window [lo, hi) of start positions so very large outputs can be
 * produced and compared piece by piece.  Both run their windows on pthreads:
 * the range is cut into blocks of BLOCK start positions, each block is
 * computed independently (a match belongs to the block of its start) and the
 * block results are concatenated in order.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define BLOCK (1u << 20)

typedef struct {
    uint64_t *pos;
    uint32_t *id;
    uint64_t n, cap;
    int oom;
} mlist;

static void ml_push(mlist *m, uint64_t p, uint32_t j) {
    if (m->oom) return;
    if (m->n == m->cap) {
        uint64_t nc = m->cap ? 2 * m->cap : 1024;
        uint64_t *np = (uint64_t *)realloc(m->pos, nc * sizeof(uint64_t));
        if (!np) { m->oom = 1; return; }
        m->pos = np;
        uint32_t *ni = (uint32_t *)realloc(m->id, nc * sizeof(uint32_t));
        if (!ni) { m->oom = 1; return; }
        m->id = ni;
        m->cap = nc;
    }
    m->pos[m->n] = p;
    m->id[m->n] = j;
    m->n++;
}

/* index of the segment containing start position p: the largest k with
 * o_k <= p and o_{k+1} > p (empty segments are skipped). */
static uint32_t seg_of(const uint64_t *seg, uint32_t n_seg, uint64_t p) {
    uint32_t lo = 0, hi = n_seg; /* answer in [lo, hi) */
    while (hi - lo > 1) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (seg[mid] <= p) lo = mid; else hi = mid;
    }
    return lo;
}

/* ---------------------------------------------------------------- O1 ---- */

typedef struct {
    const uint8_t *pat;
    const uint64_t *pat_off;
    uint32_t n;
    const uint8_t *text;
    const uint64_t *seg;
    uint32_t n_seg;
} bf_args;

static void bf_block(const bf_args *a, uint64_t lo, uint64_t hi, mlist *out) {
    if (lo >= hi) return;
    uint32_t k = seg_of(a->seg, a->n_seg, lo);
    for (; k < a->n_seg && a->seg[k] < hi; k++) {
        uint64_t s0 = a->seg[k], s1 = a->seg[k + 1];
        uint64_t p0 = s0 > lo ? s0 : lo, p1 = s1 < hi ? s1 : hi;
        for (uint64_t p = p0; p < p1; p++) {
            for (uint32_t j = 0; j < a->n; j++) {
                uint64_t L = a->pat_off[j + 1] - a->pat_off[j];
                if (p + L > s1) continue;
                if (memcmp(a->text + p, a->pat + a->pat_off[j], L) == 0) ml_push(out, p, j);
            }
        }
    }
}

/* ---------------------------------------------------------------- O2 ---- */

typedef struct oracle_ac {
    uint32_t n_nodes, cap_nodes;
    uint32_t *first_child, *next_sib, *fail, *dict, *depth;
    int32_t *out_id;
    uint8_t *sym;
    /* goto function: open-addressing hash of key (node << 8 | symbol) */
    uint64_t *hkey;
    uint32_t *hval;
    uint64_t hmask;
    uint32_t max_len;
} oracle_ac;

#define NONE 0xFFFFFFFFu
#define EMPTY 0xFFFFFFFFFFFFFFFFull

static uint64_t mix64(uint64_t x) {
    x ^= x >> 33; x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33; x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33; return x;
}

static uint32_t ac_goto(const oracle_ac *ac, uint32_t s, uint8_t c) {
    uint64_t key = ((uint64_t)s << 8) | c;
    uint64_t h = mix64(key) & ac->hmask;
    for (;;) {
        if (ac->hkey[h] == key) return ac->hval[h];
        if (ac->hkey[h] == EMPTY) return NONE;
        h = (h + 1) & ac->hmask;
    }
}

static void ac_set(oracle_ac *ac, uint32_t s, uint8_t c, uint32_t v) {
    uint64_t key = ((uint64_t)s << 8) | c;
    uint64_t h = mix64(key) & ac->hmask;
    while (ac->hkey[h] != EMPTY) h = (h + 1) & ac->hmask;
    ac->hkey[h] = key;
    ac->hval[h] = v;
}

void oac_free(oracle_ac *ac) {
    if (!ac) return;
    free(ac->first_child); free(ac->next_sib); free(ac->fail); free(ac->dict);
    free(ac->depth); free(ac->out_id); free(ac->sym); free(ac->hkey); free(ac->hval);
    free(ac);
}

/* Builds goto, failure and dictionary-suffix links.  Returns NULL on an
 * empty pattern, a duplicate pattern or allocation failure. */
oracle_ac *oac_build(const uint8_t *pat, const uint64_t *pat_off, uint32_t n) {
    uint64_t total = pat_off[n] - pat_off[0];
    uint64_t cap = total + 1;
    if (cap > 0xFFFFFFF0ull) return NULL;
    oracle_ac *ac = (oracle_ac *)calloc(1, sizeof(oracle_ac));
    if (!ac) return NULL;
    ac->cap_nodes = (uint32_t)cap;
    ac->first_child = (uint32_t *)malloc(cap * 4);
    ac->next_sib = (uint32_t *)malloc(cap * 4);
    ac->fail = (uint32_t *)malloc(cap * 4);
    ac->dict = (uint32_t *)malloc(cap * 4);
    ac->depth = (uint32_t *)malloc(cap * 4);
    ac->out_id = (int32_t *)malloc(cap * 4);
    ac->sym = (uint8_t *)malloc(cap);
    uint64_t hs = 1;
    while (hs < 2 * cap) hs <<= 1;
    ac->hmask = hs - 1;
    ac->hkey = (uint64_t *)malloc(hs * 8);
    ac->hval = (uint32_t *)malloc(hs * 4);
    if (!ac->first_child || !ac->next_sib || !ac->fail || !ac->dict || !ac->depth ||
        !ac->out_id || !ac->sym || !ac->hkey || !ac->hval) { oac_free(ac); return NULL; }
    memset(ac->hkey, 0xFF, hs * 8);

    ac->n_nodes = 1; /* root = 0 */
    ac->first_child[0] = NONE; ac->next_sib[0] = NONE; ac->depth[0] = 0;
    ac->out_id[0] = -1; ac->sym[0] = 0;
    for (uint32_t j = 0; j < n; j++) {
        uint64_t L = pat_off[j + 1] - pat_off[j];
        if (L == 0) { oac_free(ac); return NULL; }
        if (L > ac->max_len) ac->max_len = (uint32_t)L;
        uint32_t s = 0;
        for (uint64_t i = 0; i < L; i++) {
            uint8_t c = pat[pat_off[j] + i];
            uint32_t t = ac_goto(ac, s, c);
            if (t == NONE) {
                t = ac->n_nodes++;
                ac->first_child[t] = NONE;
                ac->next_sib[t] = ac->first_child[s];
                ac->first_child[s] = t;
                ac->depth[t] = ac->depth[s] + 1;
                ac->out_id[t] = -1;
                ac->sym[t] = c;
                ac_set(ac, s, c, t);
            }
            s = t;
        }
        if (ac->out_id[s] >= 0) { oac_free(ac); return NULL; } /* duplicate */
        ac->out_id[s] = (int32_t)j;
    }

    /* breadth-first failure links: fail(v) for child v of u by symbol c is
     * goto(f, c) for the first f on u's failure chain that has it, else root */
    uint32_t *queue = (uint32_t *)malloc((uint64_t)ac->n_nodes * 4);
    if (!queue) { oac_free(ac); return NULL; }
    uint32_t qh = 0, qt = 0;
    ac->fail[0] = 0; ac->dict[0] = NONE;
    for (uint32_t v = ac->first_child[0]; v != NONE; v = ac->next_sib[v]) {
        ac->fail[v] = 0; ac->dict[v] = NONE; queue[qt++] = v;
    }
    while (qh < qt) {
        uint32_t u = queue[qh++];
        for (uint32_t v = ac->first_child[u]; v != NONE; v = ac->next_sib[v]) {
            uint8_t c = ac->sym[v];
            uint32_t f = ac->fail[u], g;
            for (;;) {
                g = ac_goto(ac, f, c);
                if (g != NONE) break;
                if (f == 0) { g = 0; break; }
                f = ac->fail[f];
            }
            ac->fail[v] = g;
            /* dictionary link: nearest final state on the failure chain */
            ac->dict[v] = (ac->out_id[g] >= 0) ? g : ac->dict[g];
            queue[qt++] = v;
        }
    }
    free(queue);
    return ac;
}

typedef struct {
    const oracle_ac *ac;
    const uint8_t *text;
    const uint64_t *seg;
    uint32_t n_seg;
} ac_args;

static int cmp_match(const void *x, const void *y) {
    const uint64_t *a = (const uint64_t *)x, *b = (const uint64_t *)y;
    if (a[0] != b[0]) return a[0] < b[0] ? -1 : 1;
    if (a[1] != b[1]) return a[1] < b[1] ? -1 : 1;
    return 0;
}

static void ac_block(const ac_args *a, uint64_t lo, uint64_t hi, mlist *out) {
    if (lo >= hi) return;
    const oracle_ac *ac = a->ac;
    mlist raw = {0};
    uint32_t k = seg_of(a->seg, a->n_seg, lo);
    for (; k < a->n_seg && a->seg[k] < hi; k++) {
        uint64_t s0 = a->seg[k], s1 = a->seg[k + 1];
        uint64_t p0 = s0 > lo ? s0 : lo, p1 = s1 < hi ? s1 : hi;
        if (p0 >= p1) continue;
        /* scan far enough that every pattern starting before p1 can end */
        uint64_t e1 = p1 + (ac->max_len ? ac->max_len - 1 : 0);
        if (e1 > s1) e1 = s1;
        uint32_t s = 0;
        for (uint64_t e = p0; e < e1; e++) {
            uint8_t c = a->text[e];
            uint32_t g;
            for (;;) {
                g = ac_goto(ac, s, c);
                if (g != NONE) break;
                if (s == 0) { g = 0; break; }
                s = ac->fail[s];
            }
            s = g;
            uint32_t t = (ac->out_id[s] >= 0) ? s : ac->dict[s];
            while (t != NONE) {
                uint64_t p = e + 1 - ac->depth[t];
                if (p < p1) ml_push(&raw, p, (uint32_t)ac->out_id[t]);
                t = ac->dict[t];
            }
        }
    }
    if (raw.oom) { out->oom = 1; free(raw.pos); free(raw.id); return; }
    uint64_t *pairs = (uint64_t *)malloc((raw.n ? raw.n : 1) * 2 * sizeof(uint64_t));
    if (!pairs) { out->oom = 1; free(raw.pos); free(raw.id); return; }
    for (uint64_t i = 0; i < raw.n; i++) { pairs[2 * i] = raw.pos[i]; pairs[2 * i + 1] = raw.id[i]; }
    qsort(pairs, raw.n, 2 * sizeof(uint64_t), cmp_match);
    for (uint64_t i = 0; i < raw.n; i++) ml_push(out, pairs[2 * i], (uint32_t)pairs[2 * i + 1]);
    free(pairs); free(raw.pos); free(raw.id);
}

/* ------------------------------------------------------ thread driver ---- */

typedef struct {
    int kind; /* 1 = O1, 2 = O2 */
    const void *args;
    uint64_t lo, hi, n_blocks;
    mlist *blocks;
    uint64_t next;
    pthread_mutex_t mu;
} driver;

static void *worker(void *vp) {
    driver *d = (driver *)vp;
    for (;;) {
        pthread_mutex_lock(&d->mu);
        uint64_t b = d->next++;
        pthread_mutex_unlock(&d->mu);
        if (b >= d->n_blocks) break;
        uint64_t a = d->lo + b * (uint64_t)BLOCK, z = a + BLOCK;
        if (z > d->hi) z = d->hi;
        if (d->kind == 1) bf_block((const bf_args *)d->args, a, z, &d->blocks[b]);
        else ac_block((const ac_args *)d->args, a, z, &d->blocks[b]);
    }
    return NULL;
}

/* Runs the blocks of [lo, hi) on n_threads threads, concatenates them and
 * copies at most cap matches out.  Returns the total count, -2 on OOM. */
static int64_t drive(int kind, const void *args, uint64_t lo, uint64_t hi, int n_threads,
                     uint64_t *out_pos, uint32_t *out_id, uint64_t cap) {
    if (hi <= lo) return 0;
    driver d;
    d.kind = kind; d.args = args; d.lo = lo; d.hi = hi;
    d.n_blocks = (hi - lo + BLOCK - 1) / BLOCK;
    d.blocks = (mlist *)calloc(d.n_blocks, sizeof(mlist));
    if (!d.blocks) return -2;
    d.next = 0;
    pthread_mutex_init(&d.mu, NULL);
    if (n_threads < 1) n_threads = 1;
    if ((uint64_t)n_threads > d.n_blocks) n_threads = (int)d.n_blocks;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * n_threads);
    int started = 0;
    for (int i = 1; th && i < n_threads; i++)
        if (pthread_create(&th[started], NULL, worker, &d) == 0) started++;
    worker(&d);
    for (int i = 0; i < started; i++) pthread_join(th[i], NULL);
    free(th);
    pthread_mutex_destroy(&d.mu);
    int64_t total = 0;
    int oom = 0;
    for (uint64_t b = 0; b < d.n_blocks; b++) {
        mlist *m = &d.blocks[b];
        oom |= m->oom;
        for (uint64_t i = 0; i < m->n; i++) {
            if ((uint64_t)total < cap) { out_pos[total] = m->pos[i]; out_id[total] = m->id[i]; }
            total++;
        }
        free(m->pos); free(m->id);
    }
    free(d.blocks);
    return oom ? -2 : total;
}

/* Valid segment list: o_0 = 0, non-decreasing, o_S = N. */
static int segs_ok(const uint64_t *seg, uint32_t n_seg, uint64_t n_bytes) {
    if (n_seg == 0) return n_bytes == 0;
    if (seg[0] != 0 || seg[n_seg] != n_bytes) return 0;
    for (uint32_t k = 0; k < n_seg; k++) if (seg[k + 1] < seg[k]) return 0;
    return 1;
}

int64_t obf_match(const uint8_t *pat, const uint64_t *pat_off, uint32_t n,
                  const uint8_t *text, uint64_t n_bytes, const uint64_t *seg, uint32_t n_seg,
                  uint64_t lo, uint64_t hi, int n_threads,
                  uint64_t *out_pos, uint32_t *out_id, uint64_t cap) {
    if (!segs_ok(seg, n_seg, n_bytes)) return -1;
    for (uint32_t j = 0; j < n; j++) if (pat_off[j + 1] == pat_off[j]) return -1;
    if (hi > n_bytes) hi = n_bytes;
    if (n_seg == 0) return 0;
    bf_args a = {pat, pat_off, n, text, seg, n_seg};
    return drive(1, &a, lo, hi, n_threads, out_pos, out_id, cap);
}

int64_t oac_match(const oracle_ac *ac, const uint8_t *text, uint64_t n_bytes,
                  const uint64_t *seg, uint32_t n_seg, uint64_t lo, uint64_t hi, int n_threads,
                  uint64_t *out_pos, uint32_t *out_id, uint64_t cap) {
    if (!ac || !segs_ok(seg, n_seg, n_bytes)) return -1;
    if (hi > n_bytes) hi = n_bytes;
    if (n_seg == 0) return 0;
    ac_args a = {ac, text, seg, n_seg};
    return drive(2, &a, lo, hi, n_threads, out_pos, out_id, cap);
}

uint32_t oac_nodes(const oracle_ac *ac) { return ac ? ac->n_nodes : 0; }

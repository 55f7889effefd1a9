/*
 * pfac.h - C ABI of the GB300 failure-less Aho-Corasick (PFAC) matcher.
 *
 * The library implements exact multi-pattern matching as the paper states it
 * (Section 2.2: find every occurrence of a set of fixed patterns P in a text
 * T) with the failure-less method of Section 2.3: one walk starts at every
 * input position and follows the trie of the patterns until a symbol has no
 * transition, reporting every pattern it completes.  The trie is stored in
 * the bitmap storage model of Section 3.1 (per-node symbol bitmap, children
 * addressed by popcount rank, Eq. 1) with the leaf merge of Section 3.2
 * (Eq. 2), plus a dense lookup for the first trie levels.
 *
 * Result definition.  With distinct non-empty patterns P_0..P_{n-1} over the
 * symbols 0..sigma-1, a text T[0..N) and segment offsets
 * 0 = o_0 <= o_1 <= ... <= o_S = N, the result is the set of pairs
 *     (p, j)  with  o_k <= p,  p + |P_j| <= o_{k+1},  T[p .. p+|P_j|) = P_j
 * for some k (no occurrence crosses a segment end), sorted by p then j.
 * p is a global byte offset into T; j is the caller's index of the pattern.
 * A text byte >= sigma matches nothing (it ends every walk that reaches it).
 *
 * Output keys.  Each pair is returned as one uint64 key
 *     key = (uint64)p << PFAC_ID_BITS | j,
 * so ascending numeric order of keys is the (p, j) order.  This requires
 * n_patterns < 2^PFAC_ID_BITS and N < 2^(64 - PFAC_ID_BITS).
 *
 * Memory and streams.  Pointers named d_* are CUDA device pointers owned by
 * the caller; all other pointers are host pointers.  Every call takes the
 * CUDA stream (a cudaStream_t passed as void*, NULL = legacy default stream)
 * on which its device work is ordered.  The table is owned by the library
 * from pfac_build until pfac_table_free.  Calls on one table may run
 * concurrently on different streams as long as each uses its own workspace.
 * A table lives on the device that was current when it was built: every
 * call that launches work on it (matching, verification, autotuning,
 * serving) must be made with that device current and, when a stream is
 * given, a stream of that device; otherwise it returns PFAC_EINVAL before
 * any device work.  (While a stream captures a CUDA graph its device cannot
 * be queried, so then only the current device is checked.)
 *
 * Errors.  Every int-returning call returns a pfac_status; 0 is success.  A
 * failing call leaves its outputs unspecified (except PFAC_ENOSPC, below),
 * records a message retrievable with pfac_last_error (per host thread) and
 * never aborts the process.
 */
#ifndef PFAC_H
#define PFAC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PFAC_ID_BITS 24
#define PFAC_MAX_PATTERN_LEN (1u << 20)

typedef enum {
    PFAC_OK = 0,
    PFAC_EINVAL = -1,   /* bad argument: sizes, pointers, alignment, offsets */
    PFAC_EDUP = -2,     /* two patterns are equal */
    PFAC_ESYMBOL = -3,  /* a pattern symbol is >= alphabet_size */
    PFAC_ENOMEM = -4,   /* host or device allocation failed */
    PFAC_ENOSPC = -5,   /* output capacity too small; count reported */
    PFAC_ECUDA = -6,    /* a CUDA runtime call failed */
    PFAC_ETIMEOUT = -7, /* a bounded device wait gave up */
    PFAC_EDEVICE = -8,  /* a device-side consistency check failed */
    PFAC_EIO = -9,      /* a table file could not be opened, read or written */
    PFAC_EFORMAT = -10  /* not a table file of this format, or its checksum or
                           structure does not hold */
} pfac_status;

typedef enum {
    PFAC_LAYOUT_COMPRESSED = 0, /* bitmap trie + leaf merge + prefix table */
    PFAC_LAYOUT_DENSE = 1       /* uncompressed state-transition table */
} pfac_layout;

typedef struct pfac_table pfac_table;

/* Build options; a NULL pointer means all fields 0 (defaults). */
typedef struct {
    uint32_t layout;       /* pfac_layout */
    uint32_t prefix_depth; /* symbols resolved by the dense prefix lookup
                              (compressed layout); 0 = chosen by the library;
                              else at most 20 / b and at least 5 / b rounded
                              up, b = bits per symbol (PFAC_EINVAL otherwise) */
    uint32_t flags;        /* PFAC_BUILD_* bits */
    uint32_t truncate_depth; /* prefix matching (Section 2.4): 0 = exact
                              table; d > 0 = the trie holds every pattern's
                              first d symbols, so pfac_match reports the
                              candidates (p, j) whose first min(|P_j|, d)
                              symbols occur at p; pfac_verify keeps the exact
                              ones (the table then also keeps the patterns) */
    uint32_t reserved[4];
} pfac_build_opts;

/* Build flag: build the table on the host only (no device memory, no CUDA
 * call); the table then answers pfac_table_info but cannot match. */
#define PFAC_BUILD_HOST_ONLY 1u
/* Build flag (compressed layout): reduction step 2 of Section 3.2, equal
 * subtrees of the last three trie levels stored once (the trie becomes a
 * DAG).  A walk that stops inside a shared subtree finds its pattern ids in
 * a side table keyed by its last unshared node and the symbols after it.
 * Matches are the same; merged_trie_nodes in pfac_table_info counts the
 * nodes kept.  Such a table is matched by the queued scan kernel with its
 * prefix entries in L2 (variant 1) and 16 warps per CTA; other requests
 * return PFAC_EINVAL.  With alphabets of up to 8 symbols the merge takes the
 * packed records (not with PFAC_BUILD_WIDE_RECORDS). */
#define PFAC_BUILD_SUFFIX_MERGE 2u
/* Build flag (compressed layout, alphabets of up to 8 symbols): keep the
 * two-word records of the 32-symbol format instead of one packed word per
 * node.  Packed records are the default where the trie fits them (fewer
 * than 2^26 nodes for alphabets of up to 4 symbols, 2^22 for 5 to 8); this
 * flag exists for comparison and testing. */
#define PFAC_BUILD_WIDE_RECORDS 4u

/* Match options; a NULL pointer means library defaults (the table's
 * autotuned choice when pfac_autotune has run). */
typedef struct {
    uint32_t variant;      /* 0 = default (autotuned when pfac_autotune ran),
                              1 = prefix bitmap in shared memory, its
                              entries read through L2, 2 = prefix bitmap and
                              entries in shared memory */
    uint32_t prefix_depth; /* 0 = table default; else one the table holds */
    uint32_t ctas_per_sm;  /* 0 = default (1) */
    uint32_t bitmap_copies; /* copies of the prefix bitmap in shared memory
                              (1, 2, 4, ..., 32); 0 = as many as fit */
    void *ev_scan_begin;   /* optional cudaEvent_t recorded on the call's stream
                              right before the scan kernel, for profiling */
    void *ev_scan_end;     /* optional cudaEvent_t recorded right after it */
    uint32_t child_masks;  /* second on-chip stage (child masks of the prefix
                              entries in shared memory): 0 = when it fits,
                              1 = off, 2 = required */
    uint32_t gram_filter;  /* first on-chip stage over the table's gram filter
                              (a hashed bitmap of the g-symbol strings that
                              start a match, g = deepest prefix depth + 1)
                              instead of the prefix bitmap: 0 = when the
                              library expects it to pass fewer positions,
                              1 = off, 2 = required.  With it, bitmap_copies
                              counts copies of the gram filter. */
    uint32_t prefix_bytes; /* first on-chip stage over one byte per prefix
                              index (prefix nodes of at most 16 index bits):
                              nonzero for indices with an entry, with a
                              bucket mask of the next symbols that can follow
                              as a cheap second stage.  0 = library choice,
                              1 = off, 2 = required (one copy; excludes the
                              gram filter and bitmap_copies > 1) */
    uint32_t warps_per_cta; /* warps per CTA of the scan kernel: 0 = library
                              choice (16, or the autotuner's), 16, or 24 (80
                              registers a thread; only where the tables leave
                              shared memory for 24 warps' buffers) */
    uint64_t starts_end;   /* 0 = every input position starts a walk; else
                              only positions below it do (at most n_bytes;
                              the bytes after it are still read by walks, as
                              the halo of a shard or chunk) */
    uint64_t position_base; /* added to every reported position (a shard's
                              or chunk's global offset); position_base +
                              n_bytes must stay below 2^40 */
    void *ev_emit_begin;   /* optional cudaEvent_t recorded right before the
                              scan kernel's second (emit) launch, which
                              re-scans the slices whose matches did not fit
                              their record space, for profiling */
    void *ev_emit_end;     /* optional cudaEvent_t recorded right after it */
    uint32_t scan_kernel;  /* which scan kernel runs the first stages: 0 =
                              library choice (or the autotuner's), 1 = queued
                              kernel (input staged in shared memory by bulk
                              copies), 2 = register-staged kernel (input read
                              into registers; alphabets of 129 to 256 symbols
                              or of up to 4; excludes prefix_bytes = 2 and
                              warps_per_cta), 3 = the dense layout's
                              thread-serial kernel (one thread walks its
                              positions one after another, the transition table
                              from shared memory where it fits; for
                              comparison).  Both layouts run kernels 1 and 2,
                              the dense one over its transition table (16 warps
                              per CTA). */
    uint32_t reserved_scan;
    /* Testing aids for the failure path of the queued kernel's bounded waits
     * (they change no result of a call that does not set them): */
    uint32_t test_wait_limit_us; /* 0 = the default bound of every wait on a
                              bulk copy (4 s); else this many microseconds */
    uint32_t test_withhold_slice; /* 0 = off; s > 0: the copy of the 512-byte
                              slice s - 1 is never issued, so the wait for it
                              gives up after the bound, the kernel records
                              PFAC_ETIMEOUT (pfac_match returns it) and the
                              device stays usable */
    uint32_t records_per_slice; /* match records kept per 512-byte slice by the
                              scan pass (compressed layout): 0 = library
                              choice (512 when the pattern set makes more
                              than 8 matched positions per slice likely on
                              uniform text, else 32, or the autotuner's), 32,
                              or 512 (every position: no slice is ever scanned
                              a second time; 8 bytes of workspace per input
                              byte) */
    uint32_t resolver;     /* who resolves the scan kernel's queues of
                              survivors: 0 = library choice (the resolver
                              kernel for plain tries), 1 = the scan kernel's
                              warps themselves, 2 = the resolver kernel (a
                              second launch after the scan, which the scan's
                              warps hand whole queues to while its buffer of
                              8 entries per slice has room; about 0.27
                              workspace bytes per input byte) */
} pfac_match_opts;

typedef struct {
    uint32_t alphabet_size;
    uint32_t n_patterns;
    uint32_t min_len, max_len;
    uint32_t layout;
    uint32_t prefix_depth;     /* default prefix depth of the table */
    uint64_t trie_nodes;       /* Q: nodes of the uncompressed trie, root included */
    uint64_t trie_leaves;      /* childless nodes */
    uint64_t records;          /* node records stored after the leaf merge */
    uint64_t merged_leaves;    /* leaves folded into their parent's record */
    uint64_t device_bytes;     /* bytes of the device-resident table */
    uint64_t paper_bytes;      /* Q * (ceil(sigma/8) + 4): Section 3.1 model */
    uint64_t dense_bytes;      /* Q * 4 * sigma: one next state per symbol */
    uint64_t output_lists;     /* distinct sorted id lists */
    uint64_t output_list_words;
    uint32_t gram_len;         /* g: symbols per gram-filter string (0: none) */
    uint32_t gram_bits;        /* log2 of the gram filter's bits */
    uint64_t gram_strings;     /* g-symbol strings whose walk does something */
    uint64_t merged_trie_nodes; /* with PFAC_BUILD_SUFFIX_MERGE: nodes after
                                   reduction step 2 (unshared nodes plus one per
                                   class of equal subtrees); else 0 */
    uint64_t side_entries;     /* side-table entries of the merged trie */
    /* device_bytes by part (each part's sections, before alignment): */
    uint64_t trie_bytes;       /* node records (the dense layout: its
                                  transition table), outputs (lists, merged
                                  leaves), merged-trie indirection and side
                                  table */
    uint64_t index_bytes;      /* prefix nodes of every depth held (bitmaps,
                                  counts, entries, child masks, prefix bytes)
                                  and the gram filter; both layouts */
    uint64_t other_bytes;      /* patterns kept for verification (truncated
                                  tables) */
    uint32_t record_bytes;     /* bytes per node record (4, 8, 16 or 48; 0 for
                                  the dense layout) */
    uint32_t reserved_info;
} pfac_table_info_t;

/*
 * pfac_build - build the matching table of a pattern set (Sections 3.1, 3.2).
 *
 *   patterns[i], lengths[i]  host pointer and length of pattern i (its id);
 *                            1 <= lengths[i] <= PFAC_MAX_PATTERN_LEN, every
 *                            byte < alphabet_size.  Copied; the caller keeps
 *                            ownership.
 *   n_patterns               0 <= n < 2^PFAC_ID_BITS (0 gives an empty table)
 *   alphabet_size            1..256
 *   opts                     may be NULL
 *   cuda_stream              stream of the table upload; the call returns
 *                            after the upload completed
 *   out                      receives the table (owned by the library)
 *
 * Errors: PFAC_EINVAL (sizes, NULL pointers, empty or too long pattern),
 * PFAC_ESYMBOL, PFAC_EDUP, PFAC_ENOMEM, PFAC_ECUDA.
 */
int pfac_build(const uint8_t *const *patterns, const uint32_t *lengths, uint32_t n_patterns,
               uint32_t alphabet_size, const pfac_build_opts *opts, void *cuda_stream,
               pfac_table **out);

/*
 * pfac_workspace_bytes - device scratch needed by pfac_match_async for an
 * input of n_bytes split into n_segments segments.  Writes *bytes.  No
 * device work.  PFAC_EINVAL for n_bytes >= 2^40 (positions take 40 bits of
 * a key) or options no plan satisfies (as pfac_match).
 */
int pfac_workspace_bytes(const pfac_table *t, uint64_t n_bytes, uint32_t n_segments,
                         const pfac_match_opts *opts, uint64_t *bytes);

/*
 * pfac_match_plan - the scan configuration a pfac_match call with these
 * options would use (no device work).  Library extension: the paper has no
 * counterpart.  Fields are 0 for the uncompressed layout except smem_bytes.
 */
typedef struct {
    uint32_t variant;        /* 1 or 2, as pfac_match_opts.variant */
    uint32_t prefix_depth;   /* k */
    uint32_t bitmap_copies;  /* copies of the first-stage bitmap */
    uint32_t child_masks;    /* 1 = off, 2 = on */
    uint32_t gram_filter;    /* 1 = off, 2 = on */
    uint32_t gram_bits;      /* log2 of the bits of one shared copy of the gram filter */
    uint32_t smem_bytes;     /* dynamic shared memory per CTA of the scan kernel */
    uint32_t prefix_bytes;   /* 1 = off, 2 = on */
    uint32_t warps_per_cta;  /* warps per CTA of the scan kernel (0: uncompressed) */
    uint32_t scan_kernel;    /* 1 = queued, 2 = register-staged, 3 = thread-serial */
    uint32_t records_per_slice; /* 32 or 512 (compressed layout) */
    uint32_t resolver;       /* 1 = the scan kernel resolves its queues, 2 = the
                                resolver kernel does (0: thread-serial) */
} pfac_plan_info;
int pfac_match_plan(const pfac_table *t, const pfac_match_opts *opts, pfac_plan_info *out);

/*
 * pfac_match_async - match a device-resident text (Section 2.3), fully
 * stream-ordered: no host synchronisation, no allocation; capturable into a
 * CUDA graph.
 *
 *   d_input          n_bytes symbols; 16-byte aligned (else PFAC_EINVAL)
 *   d_seg_offsets    n_segments + 1 uint64 offsets, o_0 = 0, non-decreasing,
 *                    o_S = n_bytes (checked on the device: a violation makes
 *                    the call report PFAC_EINVAL through d_status)
 *   d_out_keys       room for out_capacity keys; the first
 *                    min(count, out_capacity) sorted keys are written
 *   d_count          device uint64: receives the total match count
 *   d_status         device int32 (may be NULL): receives PFAC_OK, PFAC_EINVAL
 *                    (bad offsets) or PFAC_EDEVICE
 *   d_workspace      pfac_workspace_bytes() bytes, 256-byte aligned, owned by
 *                    the caller; must not be shared by concurrent calls
 *
 * Host-side argument errors return PFAC_EINVAL; launch failures PFAC_ECUDA.
 */
int pfac_match_async(const pfac_table *t, const uint8_t *d_input, uint64_t n_bytes,
                     const uint64_t *d_seg_offsets, uint32_t n_segments, uint64_t *d_out_keys,
                     uint64_t out_capacity, uint64_t *d_count, int32_t *d_status,
                     void *d_workspace, uint64_t workspace_bytes, const pfac_match_opts *opts,
                     void *cuda_stream);

/*
 * pfac_match - synchronous form of pfac_match_async: allocates the workspace
 * with the stream-ordered allocator, matches, waits for the stream and writes
 * the total match count to the host *n_out.  Returns PFAC_ENOSPC when
 * count > out_capacity (the first out_capacity keys are valid and *n_out holds
 * the full count, so a second call with a larger buffer succeeds).
 */
int pfac_match(const pfac_table *t, const uint8_t *d_input, uint64_t n_bytes,
               const uint64_t *d_seg_offsets, uint32_t n_segments, uint64_t *d_out_keys,
               uint64_t out_capacity, uint64_t *n_out, const pfac_match_opts *opts,
               void *cuda_stream);

/*
 * pfac_match_host - pfac_match for a text and a result in HOST memory
 * (Section 2.3 semantics; library extension for end-to-end use: the paper
 * does not say how the text reaches the GPU or how results return).  The
 * text is cut into chunks of chunk_bytes start positions (0 = 32 MiB;
 * rounded up to 256) plus a read halo of max_len - 1 bytes; three chunks are
 * in flight at once: copies to the device, matching and the copy back of
 * keys overlap on three streams.  Each chunk is matched with
 * starts_end / position_base (pfac_match_opts), so the keys arrive in
 * global order without filtering.  Pinned host buffers (cudaHostAlloc /
 * cudaHostRegister) make the copies asynchronous; pageable ones work but
 * serialise.
 *
 *   h_input          n_bytes symbols (host; the caller keeps ownership)
 *   h_seg_offsets    n_segments + 1 uint64 offsets (host), same rules as
 *                    pfac_match (checked on the host: PFAC_EINVAL)
 *   h_out_keys       room for out_capacity keys (host); the first
 *                    min(count, out_capacity) sorted keys are written
 *   n_out            host: the total count; PFAC_ENOSPC when it exceeds
 *                    out_capacity (two-call convention as pfac_match)
 *   opts             as pfac_match; starts_end and position_base must be 0
 *   cuda_stream      the stream the matching runs on (copies use two more
 *                    streams of the library's own); the call returns after
 *                    all work completed
 *
 * Device memory for three chunks (inputs, workspaces, keys), the two copy
 * streams and pinned staging are kept per device between calls and grown on
 * demand; pfac_match_host_release frees them.  Calls from several host
 * threads are serialised.  chunk_bytes = 0 uses 32 MiB.
 */
int pfac_match_host(const pfac_table *t, const uint8_t *h_input, uint64_t n_bytes,
                    const uint64_t *h_seg_offsets, uint32_t n_segments, uint64_t *h_out_keys,
                    uint64_t out_capacity, uint64_t *n_out, uint64_t chunk_bytes,
                    const pfac_match_opts *opts, void *cuda_stream);

/*
 * pfac_verify - the secondary process of prefix matching (Section 2.4): for a
 * table built with truncate_depth d, keeps the candidate keys (p, j) whose
 * whole pattern P_j occurs at p inside p's segment (patterns of at most d
 * symbols are exact already), in the candidates' order.  The paper leaves
 * that process unspecified; this is the library's.
 *
 *   d_input, n_bytes, d_seg_offsets, n_segments   the text the candidates
 *                    came from (device; positions relative to d_input)
 *   d_keys, n_keys   candidate keys (device), as pfac_match wrote them
 *   d_out            room for n_keys keys (device); must not alias d_keys
 *   d_count          device uint64: the number of exact matches
 *
 * Stream-ordered; its scratch (about 1 byte per candidate) comes from the
 * stream-ordered allocator.  PFAC_EINVAL for a table without truncation.
 */
int pfac_verify(const pfac_table *t, const uint8_t *d_input, uint64_t n_bytes,
                const uint64_t *d_seg_offsets, uint32_t n_segments, const uint64_t *d_keys,
                uint64_t n_keys, uint64_t *d_out, uint64_t *d_count, void *cuda_stream);

/* pfac_match_host_release - free the buffers pfac_match_host keeps for the
 * current device (waits for the device first).  Library extension. */
void pfac_match_host_release(void);

/*
 * pfac_match_noalloc - pfac_match_async for callers that cannot allocate
 * device memory when they match.  (The paper has no counterpart; this is a
 * deployment aid of this library.)
 *
 * Who needs it: code that runs where an allocation is not allowed or not
 * safe, e.g. inside a custom device-memory allocator's own callbacks, in a
 * latency-critical packet loop that must never block on the allocator or
 * fail with out-of-memory halfway through a stream, or in a process whose
 * device-memory budget is fixed at start-up.  This call allocates nothing:
 * no cudaMalloc, no cudaFree, no allocating library routine.  Its scratch is
 * a device array of PFAC_NOALLOC_SCRATCH_BYTES compiled into the library,
 * which every GPU that loads the library holds until the process exits.
 *
 * Arguments are those of pfac_match_async without the workspace.  The
 * caller still provides the input, the offsets, the output keys, d_count and
 * (optionally) d_status.
 *
 * Limits and rules:
 *   - the scratch an input needs grows with its size (about 0.55 bytes per
 *     input byte, pfac_workspace_bytes gives the exact figure); where the
 *     library's own choices (512 records per slice, the resolver kernel's
 *     buffer) would not fit, the call takes 32 records per slice and the scan
 *     kernel's own resolution instead (unless the caller set both); inputs
 *     that need more than PFAC_NOALLOC_SCRATCH_BYTES even so (roughly 58 MiB
 *     of input) are rejected with PFAC_EINVAL and a message naming both
 *     sizes, before any device work;
 *   - the first call on a device looks up that device's copy of the array
 *     (cudaGetSymbolAddress, with the device current); make that first call
 *     before any stream capture.  The address is kept per device and per
 *     CUDA context: after the device's context is replaced (for example by
 *     cudaDeviceReset) the next call looks it up again, so that call too
 *     belongs before any capture;
 *   - all calls on a device share the one array, and it keeps the previous
 *     call's contents (each call clears what must start at zero), so calls
 *     whose device work overlaps in time race and give wrong results: issue
 *     them on one stream or otherwise order them.
 */
#define PFAC_NOALLOC_SCRATCH_BYTES (32u << 20)
int pfac_match_noalloc(const pfac_table *t, const uint8_t *d_input, uint64_t n_bytes,
                       const uint64_t *d_seg_offsets, uint32_t n_segments, uint64_t *d_out_keys,
                       uint64_t out_capacity, uint64_t *d_count, int32_t *d_status,
                       const pfac_match_opts *opts, void *cuda_stream);

/*
 * pfac_autotune - choose the scan configuration of a table by timing it
 * (the prefix depth resolved in shared memory, whether the prefix entries
 * live in shared memory, the child masks, the gram filter or the prefix
 * bitmap as the first stage, and how many copies of that bitmap are spread
 * over the shared-memory banks).  Each candidate runs the scan kernel
 * on the caller's device-resident sample (same argument rules as
 * pfac_match_async); the fastest becomes the table's default for later
 * pfac_match calls without options.  With a non-NULL cache_path the choice
 * is read from / appended to that text file, keyed by alphabet size,
 * pattern count, maximum pattern length, sample size class and GPU name.
 * Synchronous (waits for the stream).  out may be NULL.
 */
typedef struct {
    uint32_t variant, prefix_depth, bitmap_copies;
    uint32_t child_masks; /* 1 = off, 2 = on */
    uint32_t n_tried;
    float scan_ms;       /* scan-kernel time of the choice on the sample */
    float default_ms;    /* scan-kernel time of the library default */
    int from_cache;
    uint32_t gram_filter; /* 1 = off, 2 = on */
    uint32_t prefix_bytes; /* 1 = off, 2 = on */
    uint32_t warps_per_cta;
    uint32_t scan_kernel;  /* 1 = queued, 2 = register-staged */
    uint32_t records_per_slice;
    uint32_t resolver;     /* as pfac_match_opts.resolver (0: the library's) */
} pfac_tune_result;

int pfac_autotune(pfac_table *t, const uint8_t *d_sample, uint64_t n_bytes,
                  const uint64_t *d_seg_offsets, uint32_t n_segments, const char *cache_path,
                  void *cuda_stream, pfac_tune_result *out);

/*
 * Serving loop (continuous batching over a resident table).
 *
 * pfac_server_create starts a dispatcher thread with n_slots CUDA streams and
 * one device-memory pool of device_bytes.  pfac_server_submit queues a request
 * (host text and host segment offsets, same rules as pfac_match; both buffers
 * must stay valid until the request completes; pinned buffers make the copies
 * asynchronous).  Requests are admitted oldest first as soon as a slot is free
 * and the pool can hold the request's input, offsets, workspace and output;
 * admitted requests run concurrently on their streams.  pfac_server_wait
 * blocks until a request is done (timeout_s <= 0: no limit), pfac_server_poll
 * returns the next completed request (1 when none), and the result's keys
 * stay valid until pfac_server_release.  Keys land straight from the device
 * in a pinned host arena of host_bytes and are handed out in place; release
 * returns the block, so results released promptly keep the arena free
 * (when it is full, keys go through a staging copy into memory of their
 * own).  Times are seconds on a monotonic
 * clock: submit, admission (a slot and memory taken), issued (the host calls
 * of the admission returned), counted (the dispatcher saw the first phase
 * complete), completion.
 */
typedef struct pfac_server pfac_server;
typedef struct {
    uint32_t n_slots;           /* concurrent requests on the GPU; 0 = 4 */
    uint32_t reserved0;
    uint64_t device_bytes;      /* pool for in-flight requests; 0 = 1 GiB */
    uint64_t max_request_bytes; /* largest input accepted; 0 = device_bytes / 4 */
    uint64_t host_bytes;        /* pinned result arena; 0 = 256 MiB */
    uint64_t reserved[3];
} pfac_server_opts;
typedef struct {
    uint64_t id;
    int32_t status;             /* PFAC_OK or the request's error */
    int32_t in_arena;           /* 1: keys lie in the result arena */
    uint64_t n_keys;
    const uint64_t *keys;       /* host memory owned by the server */
    double t_submit, t_admit, t_done;
    double t_issued;            /* admission's copies and match enqueued */
    double t_counted;           /* the dispatcher saw the count (phase 1 done) */
} pfac_result;

int pfac_server_create(const pfac_table *t, const pfac_server_opts *opts, pfac_server **out);
int pfac_server_submit(pfac_server *s, const uint8_t *h_input, uint64_t n_bytes,
                       const uint64_t *h_seg_offsets, uint32_t n_segments, uint64_t *id);
int pfac_server_wait(pfac_server *s, uint64_t id, double timeout_s, pfac_result *res);
int pfac_server_poll(pfac_server *s, pfac_result *res);
int pfac_server_release(pfac_server *s, uint64_t id);
void pfac_server_destroy(pfac_server *s);

/* pfac_table_info - statistics of a built table (host call, no device work). */
int pfac_table_info(const pfac_table *t, pfac_table_info_t *out);

/*
 * pfac_table_save / pfac_table_load - checkpoint and resume of a built
 * table.  Library extension: the paper builds the compressed table once per
 * pattern set on the host and then only reads it (Section 3.1); these calls
 * let a restarted process (a serving loop, a second job) take the finished
 * table from a file instead of building it again, and let a machine without
 * a GPU build a table (PFAC_BUILD_HOST_ONLY) that a GPU machine loads.
 *
 * pfac_table_save writes t to path: a 48-byte header (magic "PFACTBL", the
 * format version, the sizes of the library's table structures, the blob's
 * bytes, a checksum), the table's description with every device pointer
 * stored as an offset into the blob, then the blob as it sits on the device
 * (read back with a synchronous copy from the table's device; host-only
 * tables write the host copy they keep).  The file is written under a
 * temporary name in the same directory and renamed over path, so a reader
 * never sees half a file.  Tuned defaults (pfac_autotune) are saved with
 * the table.  Errors: PFAC_EINVAL (NULL argument), PFAC_EIO, PFAC_ENOMEM,
 * PFAC_ECUDA.
 *
 *   pfac_table_load reads such a file and uploads the blob to the current
 *   device on cuda_stream (returning after the upload completed), or keeps
 *   it on the host when flags holds PFAC_BUILD_HOST_ONLY (the only flag
 *   accepted).  The result is the table that was saved: the same
 *   pfac_table_info, the same keys from every match call.  Checks before
 *   any allocation: the header, the checksum over description and blob
 *   (FNV-1a over 64-bit words), every field's range and every section's
 *   extent within the blob.  The contents of a section (child numbers,
 *   entries) are not checked against each other: load only files that
 *   pfac_table_save wrote.  The format holds little-endian integers and the
 *   structure sizes of this library version; a file from another version is
 *   PFAC_EFORMAT.  Errors: PFAC_EINVAL (NULL argument, unknown flag),
 *   PFAC_EIO, PFAC_EFORMAT, PFAC_ENOMEM, PFAC_ECUDA.
 */
int pfac_table_save(const pfac_table *t, const char *path);
int pfac_table_load(const char *path, uint32_t flags, void *cuda_stream, pfac_table **out);

/* pfac_table_free - releases the table's host and device memory.  The caller
 * must make sure no device work that uses the table is still pending. */
void pfac_table_free(pfac_table *t);

/* Static text of a status code. */
const char *pfac_status_str(int status);

/* Copies the calling thread's last error message (NUL-terminated, truncated
 * to n bytes) into buf; returns the status of that error (0 if none). */
int pfac_last_error(char *buf, size_t n);

/* Library version as major * 10000 + minor * 100 + patch. */
int pfac_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PFAC_H */

/*
 * ac.h -- failureless Aho-Corasick (PFAC) multi-keyword matching on NVIDIA
 * GB300 (sm_103a).  Plain C ABI: host or device pointers and sizes only.
 *
 * The problem (paper section II): locate the occurrences of any of a finite
 * set of keywords in a text.  The failureless machine used on the GPU
 * (section II, Fig. 5) has no failure transitions: every text position starts
 * its own walk through the keyword trie (section I, Fig. 3: all characters in
 * parallel) and stops at the first missing transition, so it reports, per
 * start position, only the longest keyword beginning there -- sub-pattern
 * outputs of the full machine are not reported (section II).  ac_match_full
 * adds them back: every keyword that is a prefix of a start's longest keyword
 * occurs there too, so the full machine's occurrences follow from the
 * failureless results.
 *
 * Conventions shared by every call:
 *   - Keyword ids are 0-based in the order given to ac_compile.  -1 = no match.
 *     When several keywords are the same byte string, the lowest id is reported.
 *   - Keywords and texts are raw bytes (0x00 allowed), compared exactly.
 *   - "d_" arguments are device pointers (cudaMalloc / PyTorch CUDA tensors),
 *     "h_" arguments host pointers.  `stream` is a cudaStream_t passed as void*
 *     (NULL = the legacy default stream).
 *   - Match calls are asynchronous on `stream`: they validate arguments, enqueue
 *     work and return.  Argument errors are returned synchronously.  A failure
 *     inside a kernel (a bounded wait that ran out) is latched in a per-device
 *     error word read by ac_device_status().
 *   - A handle is immutable after ac_compile and may be used from several
 *     streams at once; it must not be destroyed while work using it is in flight.
 *   - The caller owns texts and outputs; the handle owns its device tables.
 */
#ifndef AC_H
#define AC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ac_automaton *ac_handle;

typedef enum {
    AC_OK = 0,
    AC_ERR_INVALID_ARG = 1,     /* null pointer, bad size, wrong handle kind      */
    AC_ERR_EMPTY_PATTERN = 2,   /* a keyword of length 0, or k == 0               */
    AC_ERR_TOO_MANY_STATES = 3, /* more than 2^31-1 trie states                   */
    AC_ERR_OOM = 4,             /* host or device allocation failed               */
    AC_ERR_CUDA = 5,            /* a CUDA runtime call failed                     */
    AC_ERR_OVERFLOW = 6,        /* compacted output: more matches than capacity   */
    AC_ERR_BUDGET = 7,          /* request larger than the configured budget      */
    AC_ERR_TIMEOUT = 8,         /* a bounded device-side wait ran out             */
    AC_ERR_NOT_FOUND = 9,       /* unknown id (server requests)                   */
    AC_ERR_CANCELLED = 10       /* a server request cancelled before its launch   */
} ac_status;

/* Which matching kernel a handle uses (ac_set_kernel).  Results never depend
 * on the choice; only the time does. */
typedef enum {
    AC_KERNEL_TILED = 0,       /* default: bulk-copied warp tiles of text with the
                                  shared-memory root filter (a hashed filter over
                                  windows of up to 4 codes for more than 16 keyword
                                  bytes) and the survivors' walks pipelined        */
    AC_KERNEL_SIMPLE = 1,      /* one thread per position walking the goto table in
                                  global memory (the design of the paper's GPU side);
                                  ac_match and ac_match_host only                    */
    AC_KERNEL_WALK_SLOTS = 2,  /* > 16 keyword bytes: warp tiles whose survivors are
                                  walked in refilled per-lane slots (else as TILED)  */
    AC_KERNEL_THREAD_JUMP = 3, /* > 16 keyword bytes: one thread per position with the
                                  shared-memory jump table, 32 warps per SM (else as
                                  TILED)                                              */
    AC_KERNEL_THREAD_JUMP_L1 = 4 /* as THREAD_JUMP at 64 warps per SM, the jump table
                                  and the text read through L1 (else as TILED)       */
} ac_kernel;

/*
 * Build options.  Zero-initialise, or call ac_default_options.
 *   index_width    0 = choose (16-bit entries when every state id and keyword id
 *                  fits, else 32-bit), 16 or 32 to force (16 fails with
 *                  AC_ERR_INVALID_ARG when the automaton does not fit).
 *   class_compress 1 (default) = one goto column per distinct keyword byte;
 *                  0 = 256 columns (one per byte value).
 *   host_only      1 = build the host tables only; the handle can be inspected
 *                  (ac_info, ac_export_tables) but match calls refuse it.
 *                  Needs no GPU.
 *   jump_bytes     shared-memory budget of the first-level tables: the root
 *                  filter (both forms) and the root jump table of larger
 *                  alphabets; 0 = 128 KiB.
 *   stride_bytes   device budget of the second-level stride table (0 = 16 MiB;
 *                  set 1 to disable it).
 *   no_chains      1 = no chain records: every walk step reads a goto row (the
 *                  records are a speed-up only; results do not change).
 *   dev_alloc / dev_free / alloc_ctx
 *                  optional device allocator for the handle's tables (e.g. a
 *                  PyTorch caching allocator); NULL = cudaMalloc / cudaFree.
 */
typedef struct {
    int32_t index_width;
    int32_t class_compress;
    int32_t host_only;
    uint32_t jump_bytes;
    uint64_t stride_bytes;
    void *(*dev_alloc)(size_t bytes, void *ctx);
    void (*dev_free)(void *ptr, void *ctx);
    void *alloc_ctx;
    int32_t no_chains;      /* 1 = build no chain records (ac_export_chains)    */
    int32_t reserved;       /* 0                                                 */
} ac_options;

/* Shape of a compiled automaton (ac_info). */
typedef struct {
    uint32_t n_keywords;   /* k                                                     */
    uint32_t n_states;     /* trie states including the root (state 0)             */
    uint32_t n_classes;    /* goto columns used by keyword bytes                    */
    uint32_t row_width;    /* entries per goto-table row (n_classes + end column, padded) */
    uint32_t index_width;  /* bits per goto-table entry: 16 or 32                   */
    uint32_t code_bits;    /* bits per text character in the packed code stream     */
    uint32_t jump_depth;   /* characters resolved by the root jump table (k_j)      */
    uint32_t stride_depth; /* characters resolved by the stride table (0 = none)    */
    uint32_t min_len;      /* shortest keyword                                      */
    uint32_t max_len;      /* longest keyword = trie depth                          */
    uint64_t table_bytes;  /* device bytes of goto + jump + stride tables           */
    uint32_t depth_base_jump; /* first state id at depth jump_depth (BFS order)     */
    uint32_t count_jump;      /* number of states at depth jump_depth               */
    int32_t class_hash_shift; /* s when (byte >> s) & 7 tells the keyword bytes apart
                                 (at most 8 of them; bytes are then classified with
                                 byte permutes), else -1 (class table)             */
    uint32_t match_windows_ppm; /* 2- and 4-bit codes: parts per million of the
                                 jump_depth-code windows on whose walk from the root
                                 a keyword ends (from 500 on, long texts list their
                                 survivors for a second kernel by default), else 0 */
    int32_t class_direct_shift; /* 1 when the four keyword bytes have class codes
                                 (byte >> 1) & 3 (the DNA letters in either case:
                                 the kernel then takes codes from one multiply per
                                 four bytes), else -1                             */
} ac_info_t;

void ac_default_options(ac_options *opt);

/*
 * Compile a keyword set into a device-resident automaton (paper section II:
 * the goto function as a trie, stored as a matrix for the GPU, Fig. 5).
 * patterns[i] points to lens[i] bytes; the bytes are copied, so the caller may
 * free them on return.  k >= 1 and every lens[i] >= 1 (else
 * AC_ERR_EMPTY_PATTERN).  `opt` may be NULL.  Blocks until the tables are on
 * the device (the current CUDA device).  On success *out receives the handle.
 */
ac_status ac_compile(const uint8_t *const *patterns, const uint32_t *lens, uint32_t k,
                     const ac_options *opt, ac_handle *out);

/* Free a handle and its device tables.  NULL is accepted. */
ac_status ac_destroy(ac_handle h);

/* Shape of the automaton. */
ac_status ac_info(ac_handle h, ac_info_t *info);

/*
 * Copy the host tables out (for inspection and tests), any pointer may be NULL:
 *   cls   int16[256]    byte -> class code, -1 = byte in no keyword
 *   goto_ int16 or int32 [n_states * row_width]; entry > 0 = child state,
 *         entry < 0 = no transition, and the walk's result is (-entry - 2)
 *         (the longest keyword ending on the path to this state, -1 = none);
 *         column n_classes is always of the second kind (end of text)
 *   depth uint32[max_len + 1]  number of states at each depth (BFS order puts
 *         depth d at ids [sum of counts below d, ...))
 */
ac_status ac_export_tables(ac_handle h, int16_t *cls, void *goto_, uint32_t *depth);

/*
 * Chain records (for inspection and tests; host memory).  From state s_chain
 * on (BFS order), every state has a record of four uint32: a run length L
 * (0xFFFFFFFF: the state has two or more children and the walk takes its goto
 * row; 0: a leaf, the walk stops), the offset of the run's L bytes in `bytes`,
 * the state the run ends at, and the state's result (int32, -1 = none).  A
 * walk at such a state whose next L text bytes equal the run's bytes goes on
 * from the end state; otherwise it stops with the state's result (no state
 * inside a run has its own keyword).  Call with NULL arrays to get the counts
 * (*n_records, *n_bytes), then again with room for them.  s_chain = n_states
 * means no records.
 */
ac_status ac_export_chains(ac_handle h, uint32_t *s_chain, uint32_t *records, uint8_t *bytes, uint64_t *n_records,
                           uint64_t *n_bytes);

/*
 * Full-output records (for inspection and tests; host memory).  For the
 * lowest id r of each distinct keyword string (the id a walk reports), four
 * uint32 at records[4 r ..]: up = the lowest id of the longest keyword that is
 * a proper prefix of r's string (0xFFFFFFFF: none), len = |r|, dup_off, and
 * clen = the number of keyword ids that are prefixes of r's string (r's own
 * string and its equal keywords included).  dups[dup_off .. dup_off + clen -
 * clen(up)) are the ids equal to r's string, ascending.  The records of the
 * other ids are zero.  records: 4 * n_keywords entries, dups: n_keywords
 * (either may be NULL); *max_chain receives the largest clen.
 */
ac_status ac_export_full(ac_handle h, uint32_t *records, uint32_t *dups, uint32_t *max_chain);

/*
 * Root filter and window table of an automaton whose keyword bytes take 2- or
 * 4-bit codes (for inspection and tests; host memory).  A window value v holds
 * the codes of k consecutive text bytes, B bits each, the first byte lowest.
 *   F   uint32[*f_words]: the filter bit of v is bit 31 - (v & 31) of word
 *       v >> 5 (set when the walk from the root is still alive after the k
 *       bytes, or found a keyword in them); windows of fewer than 5 bits are
 *       repeated over the 32 bits of word 0.
 *   JK  int32[*jk_entries] = 2^(B k): the state reached after the k bytes, or
 *       -(result + 2) when the walk stopped inside them (result -1: none).
 * *B = 0 and zero sizes for an automaton without a filter (8-bit codes).
 * Call with NULL arrays to get the sizes, then again with room for them.
 */
ac_status ac_export_filter(ac_handle h, uint32_t *F, int32_t *JK, uint32_t *B, uint32_t *k, uint64_t *f_words,
                           uint64_t *jk_entries);

/*
 * Hashed root filter and state hash of an automaton whose keyword bytes take
 * 8-bit codes (for inspection and tests; host memory).  A window w holds the
 * codes of kh = min(4, shortest keyword) consecutive text bytes, 8 bits each,
 * the first byte lowest (a byte's code is its class, or the byte itself with
 * 256 columns).  A walk that does not reach depth kh stops before any keyword
 * ends, so its result is -1.
 *   F   uint32[2^fbits / 32]: with f = (w * 0x9E3779B1 mod 2^32) >> (32 - fbits),
 *       bit 31 - (f & 31) of word f >> 5 is set for the window of every state
 *       at depth kh (a clear bit: result -1; other windows may share a bit).
 *   HK  uint32[4 * 2^hk_bits]: entries {window, state, child, info} (state 0:
 *       empty).  The depth-kh state with window w is in the first empty entry
 *       at or after entry (w * 0x85EBCA77 mod 2^32) >> (32 - hk_bits)
 *       (cyclically), at most *probes entries from it; a window met by no
 *       entry before an empty one, or within *probes entries, has no state.
 *       child: the state's only child, 0 when it has none, 0xFFFFFFFF when it
 *       has several (or its result does not fit 24 bits); info: the child's
 *       code << 24 | (the state's result + 1), the result being the longest
 *       keyword ending on the path to the state (-1: none).
 * *kh = 0 and zero sizes for an automaton without them (2- or 4-bit codes).
 * Call with NULL arrays to get the sizes.
 */
ac_status ac_export_hash(ac_handle h, uint32_t *F, uint32_t *HK, uint32_t *kh, uint32_t *fbits, uint32_t *hk_bits,
                         uint32_t *probes);

/*
 * Stride table (for inspection and tests; host memory): for the r-th state at
 * depth k (state base_k + r, BFS order) and a window v of k2 more codes (B bits
 * each, first lowest; B as for ac_export_filter), J2[(r << (B k2)) | v] is the
 * state reached after those codes, or -(result + 2) when the walk stopped in
 * them.  *k2 = 0 and *entries = 0 when the automaton has no stride table.
 * Call with J2 = NULL to get the sizes.
 */
ac_status ac_export_stride(ac_handle h, int32_t *J2, uint32_t *k2, uint32_t *base_k, uint32_t *count_k,
                           uint64_t *entries);

/*
 * Root jump table of an automaton with 8-bit codes (for inspection and tests;
 * host memory): for a window v of k codes (8 bits each, the first byte lowest),
 * J[v] is the walk's result (>= -1) when it stopped inside the window,
 * -(2 + r) when it reached the r-th state at depth k (state base_k + r), or
 * -32768 when a result does not fit 15 bits (the kernels then walk the goto
 * table from the root).  *k = 0 and *entries = 0 without a jump table.  Call
 * with J = NULL to get the sizes.
 */
ac_status ac_export_jump(ac_handle h, int16_t *J, uint32_t *k, uint32_t *base_k, uint64_t *entries);

/*
 * Dense matching.  d_out_ids[i] = id of the longest keyword starting at
 * d_text[i] (within the n bytes), or -1.  d_text: n bytes, d_out_ids: n int32,
 * any alignment (16-byte aligned buffers take the vectorised path).  n = 0 is
 * a no-op.  Takes 16 bytes of scratch (the tile counter) per call from the
 * library's stream-ordered pool, except for a text short enough that each of
 * its tiles is some warp's first (no counter, no allocation).  A text that
 * takes the phased form of the filter kernel (8-bit codes from 4 MiB on; see
 * ac_tuning.survivor_list) also takes its survivor and walk lists from the
 * pool: about 3 bytes per text byte (16 per listed survivor, room for n / 8
 * of them, and 8 per walk).
 */
ac_status ac_match(ac_handle h, const uint8_t *d_text, uint64_t n, int32_t *d_out_ids, void *stream);

/*
 * Compacted matching: the matched start positions in ascending order with
 * their ids.  Writes min(total, cap) entries to d_pos / d_ids (uint32 each) and
 * the true total to *d_count (a device uint64).  The caller compares the total
 * with cap and calls again with more room when it is larger.  n must be below
 * 2^32.  Takes its scratch (per tile a match count, a prefix sum, 32 match
 * slots and a dense fallback of 4 bytes per position; for the phased form
 * the survivor and walk lists as for ac_match, and then no dense fallback:
 * the gather matches a tile with more than 32 matches again) from the
 * library's stream-ordered pool (cudaMallocFromPoolAsync) on `stream`; the
 * pool keeps the memory it grows to until the process exits.
 */
ac_status ac_match_compact(ac_handle h, const uint8_t *d_text, uint64_t n, uint32_t *d_pos,
                           uint32_t *d_ids, uint64_t cap, uint64_t *d_count, void *stream);

/*
 * Full Aho-Corasick output (the serial machine's output function, paper
 * section II, which reports at every text position each keyword that ends
 * there, the sub-patterns the failureless walk's longest match leaves out):
 * every occurrence of every keyword, as its end position (the index of its
 * last byte) and its id.  Entries are ordered by start position (end - len +
 * 1), then by end, then by id; equal keywords each get their own entry.
 * Writes min(total, cap) entries to d_end / d_ids (uint32 each) and the true
 * total to *d_count (a device uint64); the caller compares the total with cap
 * and calls again with more room when it is larger.  n must be below 2^32.
 * Scratch as ac_match_compact, plus 12 bytes per tile, from the same pool.
 * Returns AC_ERR_OVERFLOW when a tile's occurrences could exceed 2^32 (a
 * keyword with more than 4 million keywords among its prefixes).
 */
ac_status ac_match_full(ac_handle h, const uint8_t *d_text, uint64_t n, uint32_t *d_end, uint32_t *d_ids,
                        uint64_t cap, uint64_t *d_count, void *stream);

/* Number of matched start positions (positions whose dense id is >= 0) into
 * the device uint64 *d_count (overwritten). */
ac_status ac_count(ac_handle h, const uint8_t *d_text, uint64_t n, uint64_t *d_count, void *stream);

/*
 * Dense matching from and to HOST memory: copies h_text to the device, matches
 * and copies the ids back, pipelined in chunks on `stream` (chunks overlap
 * copies with matching; each chunk carries a max_len halo so walks never see a
 * chunk edge).  Host buffers should be pinned (cudaHostAlloc / pin_memory) for
 * the copies to overlap.  Synchronises `stream` before returning.
 */
ac_status ac_match_host(ac_handle h, const uint8_t *h_text, uint64_t n, int32_t *h_out_ids, void *stream);

/* Select the kernel used by ac_match for this handle (default AC_KERNEL_TILED). */
ac_status ac_set_kernel(ac_handle h, ac_kernel kernel);

/*
 * Launch shape of the root filter kernel (AC_KERNEL_TILED; no counterpart in
 * the paper).  Results never depend on it, only the time does.
 *   block         threads per CTA: 0 = the kernel's choice (default): 640 for
 *                 the one-phase single-text forms of 2- and 4-bit codes (20
 *                 warps per SM, compiled at 96 registers), 512 elsewhere; or
 *                 a multiple of 32, 32 .. 640 (above 512 only those forms;
 *                 the others then run at 512).
 *   stages        text tiles in flight per warp: 2 .. 4, 0 = 3 (fewer when
 *                 shared memory is short).
 *   halo          bytes bulk-copied after each tile of 992 text bytes: 0 or
 *                 16 = the look-ahead the filter's windows read (default), up
 *                 to 256 (capped at the longest keyword); the extra bytes are
 *                 not read from shared memory but reach L2 ahead of the walks
 *                 that run past the tile.
 *   per_thread    chars per thread of the one-thread-per-survivor step that
 *                 texts of 4 MiB or more with 8-bit codes take after the
 *                 filter: 2 (default; 0 means 2) or 4 survivors a thread at a
 *                 time, at 48 or 32 warps per SM.
 *   filter_bytes  shared-table depth: bytes of the root filter held in shared
 *                 memory per CTA.  ac_get_tuning reports the current size.
 *                 ac_set_tuning with a non-zero value rebuilds the root tables
 *                 for the largest filter within it, from the goto table alone:
 *                 2- and 4-bit codes, windows of k codes with 2^(B k) / 8
 *                 <= filter_bytes (and the window and stride tables for that
 *                 k); 8-bit codes, a hashed filter of 2^fbits bits, fbits
 *                 >= 5 and 2^fbits / 8 <= filter_bytes; at most 128 KiB
 *                 either way (filter_bytes below 16, or below 4 for 8-bit
 *                 codes, fits none).  0
 *                 keeps the tables.  Tables replaced stay allocated until
 *                 ac_destroy, so launches captured before still read valid
 *                 tables.  AC_ERR_INVALID_ARG for an automaton without a
 *                 root filter, or a size below the smallest filter.
 *   survivor_list how the filter kernel resolves its survivors on long single
 *                 texts (dense, count, compacted; one-launch batches and
 *                 server waves with lists follow the default rule):
 *                 0 = default (small alphabets: dense ids and counts): listed for two more kernels with 8-bit codes
 *                 (single texts from 4 MiB on), and with 2- and 4-bit codes
 *                 when at least 500 per million of the root filter's windows
 *                 already hold a match (keywords shorter than the window and
 *                 stride depth, whose many matches the warps' pipeline writes
 *                 position by position); else in the warp that filtered
 *                 them, pipelined across its tiles.  1 = listed for every
 *                 code width; 2 = always in the warp.  Small alphabets list
 *                 only beyond the texts whose heavy tiles are shared within
 *                 the CTA (about 38 MB at 512 threads on 152 SMs).
 * ac_set_tuning validates every field before changing any; do not call it
 * while work on h is being enqueued from another thread.  Batch plans and
 * servers read the tuning of their handles at each launch (a captured batch
 * graph keeps the shape it was captured with).
 */
typedef struct {
    uint32_t block;
    uint32_t stages;
    uint32_t halo;
    uint32_t per_thread;
    uint32_t filter_bytes;
    uint32_t survivor_list;
} ac_tuning;

ac_status ac_get_tuning(ac_handle h, ac_tuning *out);
ac_status ac_set_tuning(ac_handle h, const ac_tuning *t);

/*
 * Bounded waits (no counterpart in the paper).  Every wait inside this
 * handle's kernels -- a bulk copy landing on its mbarrier, an owner warp
 * waiting for the warps of its CTA to finish the rounds of a heavy tile it
 * shared, warps without work waiting for the rest of their CTA -- gives up
 * after limit_ns nanoseconds of %globaltimer (0 = the default, 2 s), latches
 * AC_ERR_TIMEOUT in the device error word (ac_device_status) and lets the
 * kernel finish; no wait spins without a limit.
 * stall_help = 1 is a test aid for the shared-tile wait: an owner warp waits
 * for one more finished round than its tile has, a count nothing ever
 * reaches, so that wait runs out after limit_ns while every round is done
 * (results stay exact).  It applies to single texts short enough to share
 * heavy tiles (ac_match, ac_count, ac_match_compact on small-alphabet
 * automata).  Do not change a handle's limit while work using it is being
 * enqueued from another thread.
 */
ac_status ac_set_wait_limit(ac_handle h, uint64_t limit_ns, int32_t stall_help);

/*
 * Compacted matching that allocates no device memory.  Same arguments, results
 * and asynchrony as ac_match_compact; the difference is where its scratch
 * lives.  ac_match_compact takes its scratch (a tile counter, per-tile counts,
 * prefix sums and match slots, and a dense fallback) from a stream-ordered pool
 * (cudaMallocFromPoolAsync) on every call; this one keeps no dense fallback and
 * matches a tile with more than 32 matches again in its gather step.  Some
 * callers cannot allocate while they match: a serving process that hands all
 * free device memory to another framework's caching allocator at start-up
 * (later cudaMalloc / cudaMallocAsync calls then fail or take memory that
 * allocator counts on), or a latency-critical loop whose rules forbid
 * allocator calls after initialisation.  This entry point uses instead one
 * file-scope device array of AC_STATIC_SCRATCH_BYTES (5 MiB) per device.
 *   - The array is committed on a device, and its device address looked up
 *     (cudaGetSymbolAddress, once per device), when the first handle is
 *     compiled there (ac_compile), and held until the process exits.  So
 *     compile before another allocator reserves the device's free memory, and
 *     before any stream capture.  A call never allocates.
 *   - Texts longer than AC_STATIC_MAX_TEXT bytes are rejected with
 *     AC_ERR_BUDGET before any work is enqueued.
 *   - Every call clears the part of the array it uses (cudaMemsetAsync on
 *     `stream`) and then launches.  All calls share the one array: calls whose
 *     work overlaps on the GPU (different streams, or host threads without
 *     ordering between them) race and give wrong results.  Serialise them.
 *   - It runs the kernel and launch shape chosen for the handle (ac_set_kernel,
 *     ac_autotune), like ac_match_compact.
 *   - The paper has no counterpart: this is a deployment variant of the
 *     compacted output.
 */
#define AC_STATIC_MAX_TEXT (16ull << 20)
#define AC_STATIC_SCRATCH_BYTES (5u << 20)
ac_status ac_match_compact_static(ac_handle h, const uint8_t *d_text, uint64_t n, uint32_t *d_pos,
                                  uint32_t *d_ids, uint64_t cap, uint64_t *d_count, void *stream);

/*
 * ---- Batches: many texts, several automata --------------------------------
 * The paper matches one text per run (section III); a batch is this library's
 * way to keep the GPU busy with many short texts: every text is cut into the
 * same work units (tiles) a single text is, and the units of all texts and all
 * automata are matched by one persistent launch (each CTA takes the automata
 * in turn, loading each one's root filter into shared memory, and its warps
 * take that automaton's units), so short texts do not each pay a launch and a
 * tail, and no launch boundary drains the GPU between automata.  That launch
 * serves up to 32 automata with root filters (every automaton has one unless
 * built with jump_bytes below 4); it runs the filter kernel for each, whatever
 * kernel ac_set_kernel or ac_autotune chose for its single texts (and, with a
 * plan's survivor lists, lists the survivors of its 8-bit-code automata, and
 * of those with 2- or 4-bit codes whose match_windows_ppm is 500 or more, for
 * two more launches: ac_batch_reserve_lists).  Otherwise the batch takes one
 * persistent launch per automaton.  Results are exactly
 * those of ac_match on each text alone: walks stop at the end of their own
 * text.
 *
 * One text of a batch: bytes d_texts[text_off, text_off + len), matched
 * against hs[automaton], dense ids written to d_out[out_off, out_off + len).
 * Texts may overlap or share bytes; their output ranges must not overlap.
 * len = 0 is allowed (nothing is written).  `reserved` must be 0.
 */
typedef struct {
    uint64_t text_off;
    uint64_t len;
    uint64_t out_off;
    uint32_t automaton;
    uint32_t reserved;
} ac_batch_item;

/*
 * Dense matching of a batch.  hs: nh handles (host array; all compiled on the
 * calling device).  d_items: nitems ac_batch_item in DEVICE memory (read by
 * the kernels; not read on the host), d_texts / d_out the bases the offsets
 * refer to.  Enqueues on `stream`: one planning kernel (groups the texts by
 * automaton and numbers their work units), then the matching launch (see
 * above).  An item whose automaton is >= nh is skipped and latches an
 * error that ac_device_status() reports as AC_ERR_INVALID_ARG.  Scratch
 * (nh * 16 + nitems * 32 bytes + 16 per automaton) comes from the library's
 * stream-ordered pool.  Asynchronous; nitems = 0 is a no-op.
 */
ac_status ac_match_batch(const ac_handle *hs, uint32_t nh, const uint8_t *d_texts, const ac_batch_item *d_items,
                         uint32_t nitems, int32_t *d_out, void *stream);

/*
 * A reusable batch plan: the handles, scratch for up to max_items texts, and
 * (after ac_batch_capture) an instantiated CUDA graph of the whole batch (the
 * planning kernel and the matching launch).
 *   ac_batch_create  copies the handle array; allocates the plan's scratch
 *                    with cudaMalloc.  max_items >= 1.
 *   ac_batch_run     enqueues the batch on `stream` (like ac_match_batch,
 *                    with the plan's scratch).  nitems <= max_items.
 *   ac_batch_capture records one ac_batch_run with these arguments into a
 *                    CUDA graph (stream capture on an internal stream) and
 *                    instantiates it, replacing any earlier graph.  Nothing
 *                    runs.
 *   ac_batch_replay  launches the captured graph on `stream`.  The pointers and
 *                    nitems are those captured; the CONTENTS of d_items (and of
 *                    the texts) may change between replays, so one graph serves
 *                    any batch of up to nitems texts over the same buffers.
 *                    AC_ERR_INVALID_ARG when nothing was captured.
 *   ac_batch_destroy frees the plan (not the handles); no work using it may be
 *                    in flight.
 *   ac_batch_reserve_lists
 *                    sizes the plan's survivor lists for the phased form of
 *                    its 8-bit-code automata (and the 2- and 4-bit ones
 *                    with match_windows_ppm of 500 or more): with the one
 *                    persistent launch,
 *                    their survivors (up to text_bytes / 8 of them per run)
 *                    are listed and resolved by two further launches at full
 *                    occupancy, as ac_match does for one long text; tiles
 *                    whose survivors no longer fit are resolved in their
 *                    warps.  Takes about 4 bytes of device memory per byte of
 *                    text_bytes (cudaMalloc); 0 frees the lists (the default:
 *                    none, every survivor is resolved in its warp).  It drops
 *                    a captured graph (capture again after it); no work
 *                    using the plan may be in flight.  Results do not depend
 *                    on it.
 * A plan must not run on two streams at once (its scratch is shared).
 */
typedef struct ac_batch_plan *ac_batch;
ac_status ac_batch_create(const ac_handle *hs, uint32_t nh, uint32_t max_items, ac_batch *out);
ac_status ac_batch_reserve_lists(ac_batch b, uint64_t text_bytes);
ac_status ac_batch_run(ac_batch b, const uint8_t *d_texts, const ac_batch_item *d_items, uint32_t nitems,
                       int32_t *d_out, void *stream);
ac_status ac_batch_capture(ac_batch b, const uint8_t *d_texts, const ac_batch_item *d_items, uint32_t nitems,
                           int32_t *d_out);
ac_status ac_batch_replay(ac_batch b, void *stream);
ac_status ac_batch_destroy(ac_batch b);

/*
 * Autotuning (no counterpart in the paper): time the dense matching of handle
 * h on the device text d_sample (n bytes, at least 1 MiB is sensible; 4 MiB or
 * more for the one-thread-per-survivor step of 8-bit codes) with each
 * candidate and keep the fastest for every later call on h (single texts,
 * batches and servers).  The candidates, for an automaton with a root filter
 * (ac_tuning): the shared-table depth -- the filter as built and two smaller
 * ones (windows of one and two codes fewer, or a hashed filter of a quarter
 * and a sixteenth of the bits) -- x threads per CTA {256, 384, 512, and 640
 * for small alphabets} x text stages {2, 3, 4} (the shapes that fit shared memory); then, at the best of
 * those, the halo (16 bytes or the longest keyword, up to 256), the survivor
 * list on and off (when the sample is long enough for it) and, with the list,
 * chars per thread {2, 4}; with 8-bit codes also the kernels
 * AC_KERNEL_THREAD_JUMP_L1, AC_KERNEL_THREAD_JUMP and AC_KERNEL_WALK_SLOTS (the
 * last with each shape).  Each candidate runs `reps` times (0 = 5) after one
 * warm-up; the median is compared.  Writes the choice to *block, *stages and
 * *kernel (an ac_kernel) when they are not NULL; ac_get_tuning reports the
 * rest.  The root tables of depths not chosen are freed.  Synchronises
 * `stream`; takes 4 * n bytes of scratch from the library pool.  Do not match
 * on h from another thread meanwhile.  Results never depend on the choice,
 * only the time does.
 */
ac_status ac_autotune(ac_handle h, const uint8_t *d_sample, uint64_t n, uint32_t reps, void *stream,
                      uint32_t *block, uint32_t *stages, uint32_t *kernel);

/*
 * ---- Serving: continuous batching of compacted-match requests ---------------
 * No counterpart in the paper.  A server keeps nh compiled automata (the
 * caller's handles, resident on the device) and a worker thread that turns the
 * stream of requests into launch waves:
 *   - a request names an automaton and a text -- in device memory (the primary
 *     path: a device-resident pool), or in pinned host memory (the secondary
 *     path: the wave copies it to the device first) -- and gets the compacted
 *     (pos, id) list of that text as ac_match_compact would give it, in caller
 *     device buffers (d_pos, d_ids, cap, d_count with the same meaning);
 *   - the HBM budget covers the resident automata (their tables, counted once
 *     per handle at ac_server_create) and the requests in flight; requests are
 *     admitted in arrival order while the bytes they hold on the device fit in
 *     what the automata leave: the text (or its device copy), 8 * cap of output
 *     and the scratch of its tiles of about 1 KiB (a match count, a prefix, 32
 *     match slots and a dense fallback of 4 bytes per position, which a tile
 *     writes only when its matches overflow the slots): about 4.4 bytes per
 *     text byte; with an automaton of 8-bit codes (in one-launch waves, below,
 *     or FIFO) 4 more per text byte for its survivor lists.  A
 *     request larger than the whole budget is refused with AC_ERR_BUDGET at
 *     submission, and a server whose automata alone exceed the budget at
 *     creation;
 *   - every admitted request that is not yet on the GPU joins the next wave:
 *     one persistent matching launch over the tiles of all its requests and
 *     automata (as a batch: up to 32 automata with root filters; else one
 *     launch per automaton), then one scan and a gather per automaton, so
 *     requests of any size share the launches.  In the one launch, when a
 *     wave holds 4 MiB or more of text for 8-bit-code automata, their
 *     survivors are listed and resolved by two more launches (the phased form
 *     of ac_match); their tiles then keep no dense fallback, and the gather
 *     matches such a tile with more than 32 matches again;
 *   - up to waves_in_flight waves run at once on their own streams: requests
 *     that arrive while a wave is on the GPU go into the next one and overlap
 *     it as SMs free up; a wave's requests complete when its last kernel ends.
 * A request's results are the same whatever else shares its wave.
 *
 * Options (zero = default):
 *   hbm_budget       device bytes of the resident automata and the admitted
 *                    requests (default 40 GiB)
 *   max_wave         most requests per wave (default 4096)
 *   waves_in_flight  waves on the GPU at once (default 2, at most 8)
 *   fifo             1 = the comparison point: one request per wave, one wave
 *                    at a time, matched by the single-text ac_match_compact path
 *   dev_alloc / dev_free / alloc_ctx
 *                    optional allocator of each wave's device scratch (plan,
 *                    host-text copies, tile scratch), e.g. a framework's caching
 *                    allocator; NULL = the library's stream-ordered pool.  A
 *                    wave's scratch is freed once the wave has completed; when
 *                    dev_alloc returns NULL the wave's requests complete with
 *                    AC_ERR_OOM.  Called from the server's worker thread.
 */
typedef struct ac_server_impl *ac_server;

typedef struct {
    uint64_t hbm_budget;
    uint32_t max_wave;
    uint32_t waves_in_flight;
    uint32_t fifo;
    uint32_t reserved;       /* 0 */
    void *(*dev_alloc)(size_t bytes, void *ctx);
    void (*dev_free)(void *ptr, void *ctx);
    void *alloc_ctx;
} ac_server_options;

/* ac_server_request.flags: the text is in pinned host memory. */
#define AC_REQ_HOST_TEXT 1u

typedef struct {
    uint32_t automaton;      /* index into the server's handles            */
    uint32_t flags;          /* 0, or AC_REQ_HOST_TEXT                     */
    const uint8_t *d_text;   /* the text (device, or pinned host with
                                AC_REQ_HOST_TEXT), n < 2^32 bytes           */
    uint64_t n;
    uint32_t *d_pos;         /* device, cap entries                        */
    uint32_t *d_ids;         /* device, cap entries                        */
    uint64_t cap;
    uint64_t *d_count;       /* device uint64: the true number of matches  */
} ac_server_request;

typedef struct {
    uint64_t ticket;         /* from ac_server_submit                      */
    int32_t status;          /* AC_OK, or why the request failed           */
    uint32_t wave_size;      /* requests in its wave                       */
    double t_submit_us;      /* host clock, microseconds since the server  */
    double t_launch_us;      /*   was created: submission, wave enqueued,  */
    double t_done_us;        /*   wave observed complete                   */
} ac_server_completion;

/* Start a server on the calling device (all handles must live there).  The
 * handle array is copied; the handles must outlive the server. */
ac_status ac_server_create(const ac_handle *hs, uint32_t nh, const ac_server_options *opt, ac_server *out);

/* Queue one request (thread-safe, returns at once).  The text and output
 * buffers must stay valid until the request completes.  n = 0 completes with
 * count 0.  AC_ERR_INVALID_ARG for a bad automaton or buffer, AC_ERR_BUDGET when
 * the request alone exceeds the budget. */
ac_status ac_server_submit(ac_server s, const ac_server_request *req, uint64_t *ticket);

/* Submit reqs[i] when the host clock reaches the call's start + arrival_us[i]
 * (non-decreasing), spinning between arrivals: a trace player for measuring
 * latency under a given arrival process.  tickets may be NULL. */
ac_status ac_server_replay(ac_server s, const ac_server_request *reqs, uint32_t n, const double *arrival_us,
                           uint64_t *tickets);

/* Move up to max completions (in completion order) to out; *n_out receives
 * how many.  wait_us > 0: wait up to that long for at least one. */
ac_status ac_server_poll(ac_server s, ac_server_completion *out, uint32_t max, uint32_t *n_out, uint32_t wait_us);

/* Block until every request submitted so far has completed (their completion
 * records stay queued for ac_server_poll). */
ac_status ac_server_drain(ac_server s);

/* Cancel a request that has not been admitted into a wave yet: it completes
 * at once with status AC_ERR_CANCELLED (its outputs are not written) and gives
 * back nothing it did not hold.  AC_ERR_NOT_FOUND when the ticket is unknown or
 * its request is already in a wave or done. */
ac_status ac_server_cancel(ac_server s, uint64_t ticket);

/* Drain, stop the worker and free the server (not the handles). */
ac_status ac_server_destroy(ac_server s);

/* Diagnostics (no counterpart in the paper): bytes of the library's
 * stream-ordered scratch pool on the calling device that are allocated now
 * (*used_now) and at most since the last reset (*used_high); reset_high = 1
 * then resets that high-water mark to the current use.  Lets a caller check
 * that a call took no pool memory (ac_match_compact_static never does). */
ac_status ac_scratch_pool_usage(uint64_t *used_now, uint64_t *used_high, int32_t reset_high);

/* Read and clear the calling device's kernel error word: AC_OK, AC_ERR_TIMEOUT
 * when a bounded wait inside a kernel ran out, or AC_ERR_INVALID_ARG when a
 * batch item named an automaton outside its handle array.  Synchronises the
 * device. */
ac_status ac_device_status(void);

/* Static description of a status code. */
const char *ac_status_string(ac_status s);

#ifdef __cplusplus
}
#endif

#endif /* AC_H */

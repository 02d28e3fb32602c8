/*
 * pfac.h — C ABI of the GB300 (sm_103a) PFAC DNA match scan.
 *
 * The method (Section IV of the paper): every text offset runs its own walk over a
 * failure-less goto trie built from the patterns, from the root, following one edge
 * per text symbol until no edge exists, and reports the id of the LONGEST pattern
 * that starts at that offset (PFAC does not report the shorter sub-patterns).
 * The trie has four columns, one per DNA base (Section V-A: a 4 x N transition
 * table); patterns are inserted one by one (Section V-A, the insertion procedure
 * after Table I). The paper's kernel runs one thread per text character and writes
 * an integer array, one entry per character (Section V-B, kernel description).
 *
 * Conventions shared by every call:
 *   - Pattern ids are 1-based in input order; 0 means "no pattern starts here".
 *     If the same string is given more than once, the lowest id is reported.
 *   - Text bytes are ASCII. Only 'A', 'C', 'G', 'T' have edges; any other byte
 *     ('N', '\n', lowercase, ...) ends every walk that reaches it. A walk never
 *     reads at or past the end of its text (or of its read, in batched calls).
 *   - Packed text: base p is stored in bits 2*(p mod 16) .. 2*(p mod 16)+1 of the
 *     32-bit word p / 16, with A=0, C=1, G=2, T=3.
 *   - Lengths and offsets are int64 (texts may exceed 2^31 bases).
 *   - Pointers named d_* are DEVICE pointers on the current CUDA device, owned by
 *     the caller (for instance torch tensors' data_ptr()); the library never frees
 *     them. A host pointer there is rejected with PFAC_ERR_INVALID_ARG: there is no
 *     CPU fallback.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Scan calls are asynchronous: the return value reports argument and launch
 *     errors only. Errors found on the device (a bad symbol met by pfac_pack, a
 *     bounded wait that ran out) are written to a status word that the caller reads
 *     after synchronising (pfac_pack's d_status, or pfac_device_status()).
 *   - Functions return PFAC_OK (0) or one of the PFAC_ERR_* codes below.
 */
#ifndef PFAC_H
#define PFAC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    PFAC_OK = 0,
    PFAC_ERR_INVALID_ARG = 1,     /* NULL or out-of-range argument, host pointer given as d_* */
    PFAC_ERR_EMPTY_PATTERN = 2,   /* a pattern of length 0 */
    PFAC_ERR_BAD_SYMBOL = 3,      /* a pattern byte (or, in pfac_pack, a text byte) outside ACGT */
    PFAC_ERR_TOO_MANY_STATES = 4, /* the trie would need 2^31 or more states */
    PFAC_ERR_OOM = 5,             /* host or device allocation failed */
    PFAC_ERR_CUDA = 6,            /* a CUDA runtime call failed (see pfac_last_cuda_error) */
    PFAC_ERR_OVERFLOW = 7,        /* more matches than the caller's capacity */
    PFAC_ERR_TIMEOUT = 8,         /* a bounded device-side wait ran out */
    PFAC_ERR_HOST_ONLY = 9,       /* the handle was built without a device copy */
    PFAC_ERR_UNSUPPORTED = 10,    /* option not available for this table (see pfac_info_ex) */
    PFAC_ERR_SCRATCH_LIMIT = 11,  /* the text is longer than pfac_match_packed_noalloc's fixed
                                     scratch buffer can serve */
    PFAC_ERR_IO = 12              /* a file cannot be opened or read */
};

/* Opaque, library-owned table handle. */
typedef struct pfac_table *pfac_handle;

/* ---------------------------------------------------------------------------
 * Table construction (Section V-A, Table I and the insertion procedure after it;
 * the breadth-first renumbering follows the state rearrangement cited in
 * Section II for cache locality).
 * ------------------------------------------------------------------------- */

/* Build the goto table from `n` patterns and upload it once to the current device.
 *   patterns[j] : host pointer to the bytes of pattern j (not NUL-terminated)
 *   lengths[j]  : its length in bytes, >= 1
 * The library copies everything it needs; the caller keeps its arrays. Sets of
 * 2 Mi bases or more are built on up to 16 host threads (one sub-trie per
 * three-base prefix, run side by side); the call returns when all of them are
 * done, and the table is the same whatever the thread count.
 * Returns NULL on error; pfac_last_error() then gives PFAC_ERR_INVALID_ARG (n <= 0
 * or a NULL array), PFAC_ERR_EMPTY_PATTERN, PFAC_ERR_BAD_SYMBOL,
 * PFAC_ERR_TOO_MANY_STATES, PFAC_ERR_OOM or PFAC_ERR_CUDA. */
pfac_handle pfac_build(const char *const *patterns, const int32_t *lengths, int32_t n);

/* Options for pfac_build_ex. Zero-initialise, then set what you need. */
typedef struct {
    int32_t host_only;  /* 1: build the tables on the host only (no device copy; the
                           scan calls reject the handle with PFAC_ERR_HOST_ONLY). */
    int32_t filter_b;   /* order of the prefix filter: 0 = automatic (about
                           log4(n) + 2.2, between 6 and 12; 14 for sets of 2^19
                           patterns or more with none shorter than 14), -1 = none,
                           1..14 = that order. One bit per b-mer, clear when a walk over
                           those b bases ends with no pattern on the way, so the answer
                           at that offset is 0 whatever follows (an exact property of
                           the same trie). A filter above order 10 (too large for shared
                           memory) comes with a first-level filter of order 10, derived
                           from it, that the packed scan keeps in shared memory. */
    int32_t sample;     /* sampled screen (see pfac_export_sample): 0 = the 13-gram
                           screen, built when the filter is of order 11 or more and every
                           pattern has at least 16 bases; 1 = that, and a 10-gram screen
                           for an order-10 filter when every pattern has at least 13 bases
                           (kept in shared memory in the filter's place by launches with
                           screen = 2; slower than the filter on genome-like texts, an
                           option for comparison); -1 = never */
} pfac_build_opts;

pfac_handle pfac_build_ex(const char *const *patterns, const int32_t *lengths, int32_t n,
                          const pfac_build_opts *opts);

/* Build the same table on the GPU from patterns already in device memory (the paper
 * builds its table on the host, Section V-A; this is the same insertion-order trie with
 * the same breadth-first numbering, computed one depth at a time: at depth d every
 * pattern longer than d marks the pair (its state, its base d), and a prefix sum over
 * the marks, state by state and base by base, numbers the new states).
 *   d_blob[...]        : DEVICE bytes of all patterns, concatenated (ASCII A/C/G/T)
 *   d_offsets[n + 1]   : DEVICE int64 offsets: pattern j is d_blob[d_offsets[j] ..
 *                        d_offsets[j + 1]); the caller guarantees they lie in d_blob
 *   opts               : as for pfac_build_ex (filter_b, sample); host_only must be 0
 *   stream             : the construction runs on it and the call returns when it is done
 * The handle's tables (rows, ids, levels, skip entries, prefix filter, rank index, dense
 * entries, first-level filter, sampled screen) equal, element for element, those of
 * pfac_build_ex on the same patterns; the handle is used and destroyed like any other.
 * Device scratch of about 20 bytes per pattern base plus 16 per pattern is allocated and
 * freed inside the call. Returns NULL on error with pfac_last_error():
 * PFAC_ERR_INVALID_ARG (n <= 0, host pointers, host_only, an offset going backwards),
 * PFAC_ERR_EMPTY_PATTERN, PFAC_ERR_BAD_SYMBOL, PFAC_ERR_TOO_MANY_STATES, PFAC_ERR_OOM or
 * PFAC_ERR_CUDA. */
pfac_handle pfac_build_device(const uint8_t *d_blob, const int64_t *d_offsets, int32_t n,
                              const pfac_build_opts *opts, void *stream);

/* File front end (the paper's host program reads its patterns and its text from files,
 * Section V-B, Figs. 4 and 5).
 *
 * pfac_build_file: build from a pattern file, as pfac_build_ex would from the same
 * patterns. One pattern per line (a trailing '\r' is dropped, empty lines are skipped);
 * a file whose first non-empty line starts with '>' is FASTA: the sequence lines of each
 * record, joined, make one pattern (ids follow the order in the file; a header with no
 * sequence line is an empty pattern, PFAC_ERR_EMPTY_PATTERN). Bytes are taken
 * as they are (no case folding), so a line holding anything but A/C/G/T fails with
 * PFAC_ERR_BAD_SYMBOL. Returns NULL on error: PFAC_ERR_IO (cannot open or read),
 * PFAC_ERR_INVALID_ARG (NULL path, no pattern) or any error of pfac_build_ex. */
pfac_handle pfac_build_file(const char *path, const pfac_build_opts *opts);

/* pfac_read_text_file: read a text file into a caller-owned HOST buffer.
 *   fasta = 0 : the bytes as they are, newlines included (a newline ends every walk
 *               that reaches it, so lines are scanned as separate reads)
 *   fasta = 1 : header lines dropped, each record's sequence lines joined, records
 *               separated by one '\n' (a record opens at a header line, or at a
 *               sequence line before the first header; one without sequence lines
 *               is an empty line of the text)
 *   *len      : receives the text's length in bytes; min(*len, cap) bytes go to buf
 *               (buf may be NULL when cap = 0: a first call that only sizes the text).
 * Returns PFAC_OK, PFAC_ERR_INVALID_ARG, PFAC_ERR_IO or PFAC_ERR_OOM. */
int pfac_read_text_file(const char *path, int32_t fasta, uint8_t *buf, int64_t cap, int64_t *len);

/* Status of the last failed call on this thread (PFAC_OK if none). */
int pfac_last_error(void);
/* Static description of a status code. */
const char *pfac_error_string(int status);
/* Text of the last CUDA runtime error seen by this thread, or "". */
const char *pfac_last_cuda_error(void);

/* Free the handle and its device memory. No launch that uses the handle may still
 * be in flight (synchronise its streams first). NULL is accepted. */
int pfac_destroy(pfac_handle h);

/* Table size: states, longest pattern, bytes held on the device. Any output may be
 * NULL. */
int pfac_info(pfac_handle h, int64_t *n_states, int32_t *max_len, int64_t *table_bytes);

typedef struct {
    int64_t n_states;       /* trie states, root included */
    int32_t n_patterns;
    int32_t max_len;        /* longest pattern = deepest level of the trie */
    int32_t min_len;
    int32_t filter_b;       /* order of the prefix filter, 0 if none */
    int64_t n_duplicates;   /* patterns whose string was given before */
    int64_t table_bytes;    /* device bytes (all layouts) */
    int64_t rows_bytes;     /* 16-byte rows: 4 x int32 per state */
    int64_t skip_bytes;     /* 16-byte skip entries, 0 if unavailable */
    int64_t filter_set;     /* b-mers whose filter bit is set (= dense entries) */
    int32_t has_skip;       /* skip entries available (fewer than 2^27 states) */
    int32_t rank_wide;      /* the filter's rank index has 32-bit entries */
    int32_t device;         /* device holding the copy, -1 if host only */
    int32_t sample_q;       /* sampled screen: q-gram length, 0 if the table has none */
    int32_t sample_s;       /* sampled screen: probe stride (see pfac_export_sample) */
    int32_t pad;
} pfac_table_info;

int pfac_info_ex(pfac_handle h, pfac_table_info *info);

/* Copy the host tables (breadth-first state order) for inspection:
 *   rows[4*S]   : rows[4*s + c] = next state for base c (A,C,G,T); bit 31 set if
 *                 that state is terminal; 0 = no edge (the root is never a target)
 *   out_id[S]   : id of the pattern ending at state s, 0 if none
 *   level[L+2]  : states of depth d are [level[d], level[d+1]) (L = max_len)
 * Any output may be NULL. S = n_states from pfac_info. */
int pfac_export(pfac_handle h, int32_t *rows, int32_t *out_id, int64_t *level);

/* Copy the device-side encodings of a handle for inspection (from the host copy of a
 * host-only handle, else from the device copy, synchronously). All three describe the
 * same trie as pfac_export (which, for a handle built by pfac_build_device, also reads
 * the device copy):
 *   skip[4*S]      : per state s, (label, meta, last, node): the chain of single-child
 *                    edges below s. meta bits 0..4 = chain length L (0..16), bit 8 = s
 *                    is terminal, bit 10 = the chain's last state is terminal; label
 *                    holds the L bases (base i in bits 2i..2i+1); last = the state L
 *                    bases below s; node = s's node word (bits 0..3 child mask, bit 4
 *                    terminal, bits 5..31 first child)
 *   filter[max(1, 4^b / 32)] : bit w (bit w mod 32 of word w / 32) of the b-mer w (base
 *                    j in bits 2j..2j+1) is clear when the walk over w ends before depth
 *                    b with no pattern on the way
 *   dense[4*F]     : one entry per set filter bit, in b-mer order: the skip entry of the
 *                    state of depth b the walk reaches, or meta bit 9 (special) when a
 *                    pattern ends within the b-mer
 * Any output may be NULL; sizes (in uint32 words) are checked against the tables. */
int pfac_export_shortcuts(pfac_handle h, uint32_t *skip, int64_t skip_words, uint32_t *filter,
                          int64_t filter_words, uint32_t *dense, int64_t dense_words);

/* Copy the sampled screen of a handle (from its host copy, or from its device copy when
 * it has one): 4^q bits (q = sample_q of
 * pfac_info_ex; bit g = bit g mod 32 of word g / 32, base j of g in bits 2j..2j+1), set
 * for the q-grams at positions 0 .. s-1 (s = sample_s) of every pattern. The builder
 * makes it for tables whose prefix filter is of order 11 or more and whose patterns all
 * have at least q + s - 1 bases; the packed scan then probes the text at every s-th
 * offset and walks only from offsets whose next probe (at or after them) is set, since
 * a pattern starting at offset i has its q-gram at position (-i) mod s at that probe.
 * `words` is the capacity of `sample` in uint32 words (0 and NULL when the table has
 * none: nothing is copied). Not in the paper: a screen of this build. */
int pfac_export_sample(pfac_handle h, uint32_t *sample, int64_t words);

/* ---------------------------------------------------------------------------
 * Launch configuration (what the autotuner chooses). All fields 0 = automatic.
 * ------------------------------------------------------------------------- */
typedef struct {
    int32_t kernel;          /* 0 auto, 1 = per-offset walk over 16-byte rows in global
                                memory (one thread per text offset, the paper's layout),
                                2 = pipelined: text staged by TMA into a shared-memory
                                ring, prefix filter and its rank index in shared memory,
                                skip-entry walks for the offsets the filter passes (needs
                                the filter and skip entries) */
    int32_t threads;         /* kernel 2: threads per CTA, 64..1024, multiple of 32: one
                                producer warp plus consumer warps */
    int32_t ctas_per_sm;     /* kernel 2: resident CTAs per SM of the persistent grid */
    int32_t stages;          /* kernel 2: text stages in the ring, 2..8 (0 = 3 for packed
                                text, 2 for ASCII) */
    int32_t rank_in_smem;    /* kernel 2: -1 = keep the filter's rank index in global
                                memory, 0 = in shared memory when it fits */
    int32_t l2_persist;      /* 1 = keep the skip entries in L2 with an access-policy
                                window, 2 = keep the prefix filter and the sampled screen
                                in L2 (tables with a sampled screen; both sit side by side
                                in the table's memory) (either sets the context's
                                persisting-L2 limit, which the next launch without a window
                                gives back; on the workloads measured both windows made the
                                scan slower), -1 or 0 = no window */
    int32_t walk_loads;      /* kernel 2: dependent table loads a walk may take before it
                                is handed to the tail kernel (0 = 2) */
    int32_t lane_offsets;    /* kernel 2: consecutive offsets per consumer lane, 16 or 32
                                (0 = 32 for packed text, 16 for ASCII and batched passes);
                                a tile is 32 x lane_offsets bases per consumer warp */
    /* Kernel 1, dense ids: the paper's memory-placement experiments (Section V-C;
     * Section VII, Figs. 6-8). Ignored by kernel 2 and by the match-list calls. */
    int32_t table_layout;    /* 0 = 16-byte rows (next state with a terminal flag) and ids by
                                state; 1 = the paper's two arrays, nextState[4 x states] and
                                matchedPatternId[4 x states] (the id of the pattern that ends
                                on the state an edge leads to); 2 = the two merged into one
                                array of (nextState, matchedPatternId) pairs, 8 bytes per
                                edge. Layouts 1 and 2 are derived on the device from the
                                rows by the pfac_set_config call that first asks for them
                                (one device allocation of 32 bytes per state, kept until
                                pfac_destroy; the call synchronises the device) */
    int32_t row_loads;       /* 0 = table loads through the read-only (texture) data path,
                                1 = default global loads, cached in L1, 2 = L1 bypassed
                                (loads cached in L2 only: the paper's L1-off setting) */
    int32_t text_smem;       /* 1 = each 256-thread block first copies its text (its 256
                                offsets plus max_len - 1 bases) into shared memory and
                                walks from there; tables whose tile would exceed 48 KB fall
                                back to reading the text from global memory */
    int32_t zero_writer;     /* kernel 2, dense ids of packed text with 32 offsets per lane:
                                who stores the ids of offsets without a match (most of the
                                output): 0 = automatic, 1 = each consumer warp stores its
                                own, 2 = one warp of the CTA stores them all with 16-byte
                                stores, 3 = one warp stores them with TMA bulk copies of a
                                zero tile in shared memory, 4 = each consumer warp stores its
                                own with TMA bulk copies of that tile. With 2 and 3 the
                                consumer warps store a match only after the writer has
                                published that its tile's zeros are written; with 4 a warp
                                stores the matches of a tile only once that tile's bulk
                                copies have completed. */
    int32_t screen;          /* kernel 2, packed text, prefix filter too large for shared
                                memory: which screen picks the offsets whose filter bit is
                                read from global memory: 0 = automatic (the sampled screen
                                when the table has one, else the first-level filter),
                                1 = the order-10 first-level filter in shared memory, 2 = the
                                sampled screen (pfac_export_sample; 32 offsets per lane); for a
                                table with an order-10 filter and a 10-gram screen, 2 = that
                                screen in shared memory in the filter's place */
    int32_t reserved;        /* 0 */
} pfac_config;

/* Set (cfg != NULL) or reset (cfg == NULL) the launch configuration of a handle.
 * Takes effect for launches issued afterwards. Out-of-range fields give
 * PFAC_ERR_INVALID_ARG and leave the previous configuration in place; asking for
 * table_layout 1 or 2 on a handle with a device copy builds that layout first (device
 * memory; PFAC_ERR_OOM or PFAC_ERR_CUDA if that fails). */
int pfac_set_config(pfac_handle h, const pfac_config *cfg);
/* The configuration the next packed-text launch on `n_bases` bases would use (an ASCII
 * launch differs only where the set configuration leaves stages or lane_offsets at 0:
 * it then uses 2 stages and 16 offsets per lane). */
int pfac_get_config(pfac_handle h, int64_t n_bases, pfac_config *cfg);

/* ---------------------------------------------------------------------------
 * Scans (Section IV; Section V-B).
 * ------------------------------------------------------------------------- */

/* 2-bit packing of ASCII text (not in the paper, which reads characters).
 *   d_text[len]            : ASCII bases
 *   d_packed[(len+15)/16]  : output words (layout above); bases past len are 0
 *   d_status (may be NULL) : int32 set to PFAC_OK, or PFAC_ERR_BAD_SYMBOL if some
 *                            byte is outside ACGT (such a byte is packed as A)
 *   d_bad (may be NULL)    : int64 set to the first such offset, or -1
 * d_status and d_bad are reset by the call itself (stream-ordered). */
int pfac_pack(const uint8_t *d_text, int64_t len, uint32_t *d_packed, int32_t *d_status,
              int64_t *d_bad, void *stream);

/* Longest-pattern id for every offset of an ASCII text: d_out_ids[i], i in [0, len). */
int pfac_match(pfac_handle h, const uint8_t *d_text, int64_t len, int32_t *d_out_ids,
               void *stream);

/* The same on packed text (n_bases bases in d_packed[(n_bases+15)/16]). */
int pfac_match_packed(pfac_handle h, const uint32_t *d_packed, int64_t n_bases,
                      int32_t *d_out_ids, void *stream);

/* Match list instead of a dense array: for every offset i with a non-zero id,
 * one (d_offsets[k], d_ids[k]) pair, k < capacity, in no particular order.
 * *d_count receives the total number of matches. When that exceeds capacity, only
 * `capacity` pairs are written (which ones is unspecified), and the kernel records
 * PFAC_ERR_OVERFLOW in the handle's device status word: pfac_device_status() returns
 * it after the launch (the call itself is asynchronous, so its return value cannot).
 * d_count is reset by the call itself (stream-ordered). Lanes of a warp that find
 * matches together take their places in the list with one atomic add. */
int pfac_match_compact(pfac_handle h, const uint32_t *d_packed, int64_t n_bases,
                       int64_t *d_offsets, int32_t *d_ids, int64_t capacity,
                       int64_t *d_count, void *stream);

/* Every pattern occurrence, not only the longest per offset: for every offset i and
 * every distinct pattern string that starts at i, one (d_offsets[k], d_ids[k]) pair with
 * that string's lowest id, k < capacity, in no particular order. This is the walk of
 * Section IV reporting each terminal state it passes, the sub-patterns included that the
 * paper's PFAC leaves out (it lists what classic Aho-Corasick, Section III, finds, with
 * occurrences keyed by their start). Same arguments, overflow rule and d_count reset as
 * pfac_match_compact. */
int pfac_match_all(pfac_handle h, const uint32_t *d_packed, int64_t n_bases,
                   int64_t *d_offsets, int32_t *d_ids, int64_t capacity,
                   int64_t *d_count, void *stream);

/* Many reads against many resident tables in ONE pass (not in the paper, whose input
 * is newline-separated reads scanned as one text, Table IV).
 *   sets[n_sets]                 : host array of handles built on this device
 *                                  (1 <= n_sets <= 65535)
 *   d_texts[text_len]            : all reads' ASCII bytes, concatenated
 *   d_read_offsets[n_reads + 1]  : read r is d_texts[off[r] .. off[r+1]) (offsets are
 *                                  clamped to [0, text_len]; a read with off[r+1] <=
 *                                  off[r] is empty). Reads should not overlap; where two
 *                                  do, each offset of the overlap gets the result of one
 *                                  of them, which one is unspecified.
 *   d_read_set[n_reads]          : index into sets[] of the table for read r
 *   d_out_ids[text_len]          : same layout as d_texts; every offset inside a read
 *                                  gets the longest pattern starting there, within the
 *                                  read (offsets outside every read are not written)
 * Walks never cross a read's end; bytes outside ACGT end walks as in pfac_match. A
 * read_set entry outside [0, n_sets) records PFAC_ERR_INVALID_ARG in the device status
 * of sets[0] and leaves that read's output unwritten.
 * Up to 8,192 reads the call is ONE kernel launch on
 * `stream`: every CTA plans the batch in shared memory (reads grouped by table), scans
 * the work items dealt to it straight from the ASCII bytes, and finishes the few long
 * walks its items deferred. Larger batches take four launches (pack the text, plan the
 * work items, one persistent scan, a tail for the long walks). Scratch (the list of
 * deferred walks; for large batches also the packed text and the plan) is kept by the
 * library per stream. The launch shape comes from the configuration of sets[0]
 * (pfac_set_config): a work item is 32 x lane_offsets offsets of one read, the scan
 * runs threads x ctas_per_sm threads per SM (one CTA per SM of up to 1,024 threads in
 * the one-launch pass; 256-thread blocks, 1 to 8 per SM, otherwise), and walk_loads
 * bounds the in-kernel walks as in kernel 2. The first call with a given list of handles uploads a small
 * descriptor array, and the first call on a stream (or with a larger text) allocates
 * scratch; both are synchronous, so issue such a call before capturing the stream
 * into a CUDA graph; later calls with the same handle list and sizes are capturable. */
int pfac_match_batched(const pfac_handle *sets, int32_t n_sets, const uint8_t *d_texts,
                       int64_t text_len, const int64_t *d_read_offsets, const int32_t *d_read_set,
                       int32_t n_reads, int32_t *d_out_ids, void *stream);

/* Read (and clear) the device status word of a handle: PFAC_OK or the first error a
 * kernel recorded since the last read (PFAC_ERR_TIMEOUT from a bounded wait,
 * PFAC_ERR_OVERFLOW from a match list that ran out of capacity, PFAC_ERR_INVALID_ARG
 * from a batched read naming a table that does not exist). Synchronises `stream`. */
int pfac_device_status(pfac_handle h, int32_t *status, void *stream);

/* ---------------------------------------------------------------------------
 * Allocation-free scan (the paper has no counterpart).
 * ------------------------------------------------------------------------- */

/* pfac_match_packed without any device allocation by the library, for callers that
 * cannot have device memory allocated on their behalf: processes that run under a
 * fixed device-memory budget or whose device memory belongs to another allocator
 * (a framework's caching pool), and latency-sensitive loops that must not meet the
 * device-wide synchronisation a cudaMalloc or cudaFree can cause.
 *
 * The ordinary scan keeps its list of deferred long walks in scratch that the library
 * allocates per stream on first use. This entry point uses instead one fixed buffer
 * compiled into the library (6 MiB, 2^18 deferred walks), which every GPU that loads
 * the library holds until the process exits. Arguments, output and results are those
 * of pfac_match_packed; the caller still passes the text and the output.
 *   - n_bases may be at most 2^26 (67,108,864 bases): longer texts are rejected with
 *     PFAC_ERR_SCRATCH_LIMIT before anything is launched (split them into pieces that
 *     overlap by max_len - 1 bases).
 *   - The first call on a device looks up the buffer's device address with that device
 *     current; make that first call before capturing any stream.
 *   - All calls share the one buffer and each call clears the part that must start at
 *     zero: calls that overlap on the GPU (on different streams, or from several host
 *     threads without ordering) race on it and must not be issued. */
int pfac_match_packed_noalloc(pfac_handle h, const uint32_t *d_packed, int64_t n_bases,
                              int32_t *d_out_ids, void *stream);

/* ---------------------------------------------------------------------------
 * Failure detection (the paper has no counterpart).
 * ------------------------------------------------------------------------- */

/* Launch a one-CTA kernel that waits on an mbarrier nothing ever completes, with the
 * same bounded wait the scan kernels use for their TMA copies. After limit_ns
 * nanoseconds the wait gives up and PFAC_ERR_TIMEOUT is written to *d_status (an
 * int32 device word; the call resets it first). Lets a test check that a wait which
 * runs out leaves the context usable and reports an error status, without faulting
 * or hanging the GPU. */
int pfac_debug_timeout_probe(int32_t *d_status, int64_t limit_ns, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PFAC_H */

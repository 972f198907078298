/*
 * ss_sort — string sample sort with LCP output on one NVIDIA GB300 (sm_103a).
 *
 * The library sorts n strings and returns their sorted order and LCP array,
 * following the problem statement of Section 2.1 of Bingmann, "Scalable String
 * and Suffix Sorting" (arXiv:1808.00963): the input is an array of n strings
 * over the alphabet {1..255}, each ending at a zero byte; the output is the
 * lexicographic order and the LCP array H with H[i] = lcp(s_{i-1}, s_i).
 * The method is the data-parallel step of Super Scalar String Sample Sort
 * (Algorithm 4.1, Section 4.2.2) and its parallel form (Section 4.2.8).
 *
 * Data layout (all data pointers are DEVICE pointers owned by the caller; the
 * library never frees them):
 *   chars      uint8[N]   NUL-terminated strings; strings may overlap (e.g.
 *                         all suffixes of one text).  Any alignment.
 *   offsets    uint64[n]  string i starts at chars + offsets[i].
 *   out_perm   uint32[n]  written: out_perm[j] = index of the j-th smallest
 *                         string.  Equal strings keep ascending index order,
 *                         so the output is unique.
 *   out_lcp    uint32[n]  written (may be NULL to skip): out_lcp[0] = 0 and
 *                         out_lcp[j] = length of the common prefix of strings
 *                         out_perm[j-1] and out_perm[j].  Two equal strings
 *                         have lcp = their length.
 * Reads of a string stay inside the 4 KiB-aligned blocks that hold a byte of
 * the string or its terminator: the library loads aligned 8-byte words, and
 * when it looks ahead along a long common prefix it may read bytes past a
 * terminator inside such a block (they are ignored).  Memory is mapped in
 * blocks of at least 4 KiB, so these reads never leave mapped memory.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  All work is enqueued on it.
 *
 * Errors: argument errors are returned at once, before any work is enqueued.
 * Errors found on the device (a bounded wait that expired, a string longer
 * than 2^30 bytes) are latched in a device status word: the asynchronous
 * calls (ss_sort, ss_sort_ex, ss_batch_run) leave it to be read by
 * ss_stream_status() / ss_batch_status(); the calls that wait for their
 * result (ss_sort_host, ss_sort_dna, ss_suffix_array, ss_sort_batch,
 * ss_sort_noalloc) return it.  A sort that latched a device-side error writes
 * the identity permutation and zero LCPs to its outputs, so that no index in
 * them is out of range.
 */
#ifndef SS_SORT_H
#define SS_SORT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ss_status {
    SS_OK = 0,
    SS_ERR_INVALID = 1,     /* bad argument (NULL pointer with n > 0, bad option) */
    SS_ERR_OOM = 2,         /* device or pinned memory could not be allocated     */
    SS_ERR_CUDA = 3,        /* a CUDA runtime call failed                         */
    SS_ERR_TOO_LARGE = 4,   /* n >= 2^32, or a string of 2^30 bytes or more       */
    SS_ERR_TIMEOUT = 5,     /* a device-side bounded wait expired                 */
    SS_ERR_QUEUE_FULL = 6,  /* a device task list overflowed its capacity (every
                               list is sized by an exact bound on its tasks, so
                               this reports an internal inconsistency)        */
    SS_ERR_NO_DEVICE = 7    /* no CUDA device, or the device is not sm_103        */
} ss_status;

/* Tuning and limits.  Zero in any field selects the default. */
typedef struct ss_options {
    uint32_t max_len;          /* 0: strings end at their NUL.  Else string i also
                                  ends after max_len bytes: a byte at position
                                  >= max_len reads as the terminator.           */
    uint32_t splitters_log2;   /* d with v = 2^d - 1 splitters per step in the
                                  single-block steps; 7..10 (default 8).        */
    uint32_t big_splitters_log2; /* d for the multi-block steps (16-character keys);
                                  8..9 (default 9).                              */
    uint32_t tile_rounds;      /* multi-block tile = 256 * tile_rounds strings;
                                  8..32 (default: chosen per step from the
                                  number of strings in big subsets).            */
    uint32_t small_cutoff;     /* subsets of at most this many strings are
                                  finished in shared memory; 64..4096
                                  (default 1024).                               */
    uint32_t big_threshold;    /* subsets larger than this use multi-block
                                  steps; >= small_cutoff (default 8192).         */
    uint32_t seed;             /* seed of the splitter sample (output does not
                                  depend on it).                                */
    uint32_t classifier;       /* classification variant of Section 4.2.3 (the
                                  output does not depend on it): 0 = S5-UI,
                                  unrolled <=-descent then one equality test
                                  against the sorted splitters (default);
                                  1 = S5-UIC, the same test done in the tree
                                  through Lemma 4.1's index map; 2 = S5-E, an
                                  equality test at every node; 3 = S5-UI
                                  entered through a jump table over the key's
                                  top 12 bits (Section 4.4; multi-block steps,
                                  the others as 0).                             */
    uint32_t host_parts;       /* ss_sort_host only: the strings are cut into
                                  this many parts by index, and part p is
                                  sorted while part p + 1 is still being
                                  copied; the sorted parts are LCP-merged
                                  (Section 4.3).  0 or 1 = copy everything,
                                  then sort (the default: over a host link
                                  as fast as the sort, the parts' sorts and
                                  merges cost more than the overlap saves);
                                  else a power of two <= 16.  Ignored
                                  elsewhere.                                  */
    uint32_t wait_limit_us;    /* bound, in microseconds, on every device-side
                                  wait of the sort (a block waiting for the
                                  work queue's next task or for a queue slot
                                  to be read); when one expires the sort
                                  stops with SS_ERR_TIMEOUT and its outputs
                                  hold the identity permutation and zero
                                  LCPs (default 30 s).  Lets a caller
                                  that must not hang detect a stalled device
                                  sooner.  An idle block of the work-queue
                                  kernel waits while other blocks split the
                                  subsets that will feed it, so a limit far
                                  below the sort's own duration stops ordinary
                                  sorts too.                                  */
    void* workspace;           /* optional caller-owned device workspace of at
                                  least ss_workspace_size() bytes, 256-byte
                                  aligned.  NULL: the library allocates
                                  stream-ordered memory for the call.           */
    size_t workspace_bytes;
} ss_options;

/* Sort n strings.  Section 2.1 (problem), Algorithm 4.1 (one S^5 step),
 * Section 4.2.8 (parallel S^5 and the LCP array).  Asynchronous: enqueues the
 * sort on `stream` and returns without waiting for it.  The rounds of
 * multi-block steps (subsets above the big threshold) are planned on the
 * device and run as one CUDA graph launch with a conditional WHILE node (one
 * graph per stream, built on the first such call); the rest is a fixed
 * sequence of launches.  The return value reports argument and launch errors;
 * device-side errors go to the stream's status word (ss_stream_status).
 * The first call on a stream allocates that stream's status word and loop
 * control block (4 KiB, kept until exit).  Without a caller workspace the
 * workspace is stream-ordered memory, freed on `stream` after the sort.
 * The caller's buffers must stay valid until the stream has run the sort.
 * n = 0 is a no-op; n = 1 gives perm = [0], lcp = [0].  Returns
 * SS_ERR_TOO_LARGE for n >= 2^32. */
ss_status ss_sort(const uint8_t* chars, const uint64_t* offsets, uint64_t n,
                  uint32_t* out_perm, uint32_t* out_lcp, void* stream);

/* ss_sort with options (opt may be NULL). */
ss_status ss_sort_ex(const uint8_t* chars, const uint64_t* offsets, uint64_t n,
                     uint32_t* out_perm, uint32_t* out_lcp, const ss_options* opt,
                     void* stream);

/* Device workspace (bytes) that ss_sort_ex needs for n strings with these
 * options (opt may be NULL). */
size_t ss_workspace_size(uint64_t n, const ss_options* opt);

/* Same as ss_sort_ex, but chars / offsets / outputs are HOST buffers:
 * chars_len bytes of chars and n offsets are copied to the device, sorted,
 * and the results copied back, all inside the call (pinned host buffers make
 * the copies fastest).  The device buffers are stream-ordered allocations
 * from the device's default memory pool, returned to the pool at the end of
 * the call.
 * With more than one part (ss_options.host_parts) the offsets are copied
 * first, then the characters part by part on a second stream, and part p is
 * sorted as soon as its characters are in (the scheme of Section 4.3.1:
 * sort parts independently, then K-way LCP-merge them).  That needs the
 * strings packed in index order (string i lies in [offsets[i],
 * offsets[i + 1]) with its terminator at offsets[i + 1] - 1, the last one
 * ending at chars_len - 1), which is checked on the device once all bytes
 * are in; a set that is not packed that way (overlapping strings, gaps,
 * another order) is then sorted again as a whole, with the same result.
 * offsets must then be host-readable memory (SS_ERR_INVALID for a device
 * pointer).  The extra device memory of the parts is 64 bytes per string. */
ss_status ss_sort_host(const uint8_t* chars, uint64_t chars_len, const uint64_t* offsets,
                       uint64_t n, uint32_t* out_perm, uint32_t* out_lcp,
                       const ss_options* opt, void* stream);

/* ss_sort_ex for strings over the DNA alphabet, with alphabet compression
 * (Section 4.4, "Alphabet compression"): chars[0, chars_len) (DEVICE) holds
 * only the bytes 'A', 'C', 'G', 'T' and the zero terminator; it is packed
 * into 3-bit codes (terminator, A, C, G, T), so that each key of the sort
 * holds 21 characters instead of 8.  Same output as ss_sort_ex on the same
 * strings (A < C < G < T as bytes).  A device copy of 3 bits per byte of
 * chars is allocated from the stream-ordered pool for the call.  Returns
 * SS_ERR_INVALID (after the call has run; the outputs are then undefined) if
 * another byte occurs in chars[0, chars_len); otherwise as ss_sort_ex. */
ss_status ss_sort_dna(const uint8_t* chars, uint64_t chars_len, const uint64_t* offsets, uint64_t n,
                      uint32_t* out_perm, uint32_t* out_lcp, const ss_options* opt, void* stream);

/* Distinguishing characters and prefixes of a sorted set (the outputs of
 * ss_sort on the same strings and max_len).  For each sorted position j,
 * with h_j = lcp[j] (h_0 = 0) and h_n = 0:
 *   out_char[j]    = c^_j = s_j[h_j], the character at which the string first
 *                    differs from its predecessor (0 if it ends there) — the
 *                    cached character of the LCP merge's caching variant
 *                    (Section 4.3.4);
 *   out_dprefix[j] = d_j = max(h_j, h_{j+1}) + 1, the length of its
 *                    distinguishing prefix (proof of Lemma 2.1);
 *   *out_D        += sum_j d_j = D (out_D: a device uint64).
 * Any output may be NULL (chars/offsets are only read for out_char).
 * Asynchronous on `stream`; argument errors are returned at once. */
ss_status ss_distinguishing(const uint8_t* chars, const uint64_t* offsets, uint64_t n, uint32_t max_len,
                            const uint32_t* perm, const uint32_t* lcp, uint8_t* out_char,
                            uint32_t* out_dprefix, uint64_t* out_D, void* stream);

/* ---- K-way LCP merge of sorted runs ----------------------------------------- */

/* Up to this many runs per ss_merge call. */
#define SS_MERGE_MAX_RUNS 64

/* One sorted run of strings of the set (chars, offsets) given to ss_merge
 * (device pointers, owned by the caller). */
typedef struct ss_run {
    const uint32_t* perm;      /* n string indices, in string order with equal
                                  strings in ascending index order (as ss_sort
                                  writes them, mapped to the set's indices).  */
    const uint32_t* lcp;       /* lcp[j] = lcp(perm[j-1], perm[j]) for j >= 1
                                  (lcp[0] is not read), as ss_sort writes it.  */
    uint32_t n;
    uint32_t reserved;         /* must be 0 */
} ss_run;

/* Merge K sorted runs into one sorted sequence with its LCP array: the
 * multiway LCP-merge of Section 4.3.2, done as ceil(log2 K) rounds of binary
 * LCP merges (LCP-Compare, Algorithm 4.2; Algorithms 4.3 and 4.4), each split
 * into independent pieces as in Section 4.3.3.
 *   runs       HOST array of num_runs (1..SS_MERGE_MAX_RUNS) run descriptors;
 *              read during the call only.  Every index must be < the number
 *              of strings behind offsets (not checked).  An index may appear
 *              in several runs: it is then output once per appearance.
 *   offsets    as for ss_sort; every offset must be below 2^56 (not checked:
 *              the merge's records keep a count in the offset's top byte).
 *   out_perm   uint32[total] (total = sum of the runs' n): the union of the
 *              runs in string order, equal strings by ascending index — the
 *              result of sorting the union with ss_sort.
 *   out_lcp    uint32[total] or NULL: out_lcp[0] = 0, out_lcp[j] = lcp of
 *              out_perm[j-1] and out_perm[j].
 *   max_len    as ss_options.max_len; it must be the value the runs were
 *              sorted with.  Strings are compared up to 2^30 characters.
 *   sample_step  every sample_step-th string of a run bounds a piece
 *              (16..65536; 0 = 64).
 *   workspace  device memory of ss_merge_workspace_size() bytes, 256-byte
 *              aligned, or NULL (a stream-ordered allocation is made and
 *              freed on `stream`).
 * Asynchronous on `stream` (no host synchronisation; no device status word:
 * the result is defined when the inputs meet the conditions above).  Output
 * buffers must not overlap the runs.  Returns SS_ERR_INVALID for bad
 * arguments, SS_ERR_TOO_LARGE if total >= 2^32 - 1, SS_ERR_OOM if the
 * workspace cannot be allocated. */
ss_status ss_merge(const uint8_t* chars, const uint64_t* offsets, uint32_t max_len,
                   const ss_run* runs, uint32_t num_runs, uint32_t sample_step,
                   uint32_t* out_perm, uint32_t* out_lcp,
                   void* workspace, size_t workspace_bytes, void* stream);

/* Workspace bytes ss_merge needs for these runs: two 32-byte records per
 * string, plus the sample counts (256 for a single run; 0 for invalid
 * arguments). */
size_t ss_merge_workspace_size(const ss_run* runs, uint32_t num_runs, uint32_t sample_step);

/* ---- suffix array by prefix doubling ---------------------------------------- */

/* Suffix array (and LCP array) of a text, by prefix doubling on top of the
 * string sort (Section 8.2: Observation 8.1, Algorithms 8.1 and 8.3).  Round
 * 0 sorts all suffixes by their first `initial_depth` characters (the string
 * sort with that cap; 0 = 256, at most 2^20); every later round sorts only the
 * suffixes of groups that are still tied, by the name pair of Observation
 * 8.1, doubling the sorted depth, until every group is a single suffix.
 *   text     DEVICE pointer to n bytes in 1..255 followed by a zero byte
 *            (text[n] = 0).
 *   out_sa   uint32[n] (device): out_sa[j] = start of the j-th smallest
 *            non-empty suffix (the empty suffix at n is not listed).
 *   out_lcp  uint32[n] (device) or NULL: out_lcp[0] = 0, out_lcp[j] = lcp of
 *            the suffixes out_sa[j-1] and out_sa[j].
 * Synchronous: waits for the result (the host reads the number of unsorted
 * suffixes after each round).  Device memory of about 63 bytes per text
 * character is taken from the stream-ordered pool for the call, plus, with
 * an LCP output, 4 bytes per character for every round (the names of each
 * round: an LCP above initial_depth is found by descending through them,
 * O(rounds + initial_depth / 256) per entry however long it is).  Returns
 * SS_ERR_TOO_LARGE for n >= 2^32 - 2, SS_ERR_INVALID for NULL pointers or
 * initial_depth > 2^20. */
ss_status ss_suffix_array(const uint8_t* text, uint64_t n, uint32_t* out_sa, uint32_t* out_lcp,
                          uint32_t initial_depth, void* stream);

/* ---- batched sorting: many independent string sets in one launch ----------- */

/* One string set of a batch (device pointers, as for ss_sort). */
typedef struct ss_set {
    const uint8_t* chars;
    const uint64_t* offsets;
    uint32_t n;
    uint32_t max_len;          /* per-set cap, as ss_options.max_len */
    uint32_t* out_perm;
    uint32_t* out_lcp;         /* may be NULL */
} ss_set;

typedef struct ss_batch ss_batch; /* opaque plan */

/* Plan a batch: validates the sets, uploads their descriptors and reserves
 * the device workspace (the caller's, via opt->workspace, or the library's).
 * Synchronous.  The total number of strings over all sets must be < 2^32. */
ss_status ss_batch_create(const ss_set* sets, uint32_t num_sets, const ss_options* opt,
                          ss_batch** out);

/* Device workspace (bytes) that a batch of these sets needs. */
size_t ss_batch_workspace_size(const ss_set* sets, uint32_t num_sets, const ss_options* opt);

/* Enqueue the sort of every set of the batch on `stream`.  Asynchronous: no
 * host synchronisation.  Sets above the big threshold take multi-block
 * steps, run by the loop of ss_sort: the stream's loop graph over the
 * stream's control block (allocated by the first such call on the stream),
 * or, when `stream` is being captured, the same loop over the batch's own
 * control block, added to the caller's graph (no allocation then).  The rest
 * is a fixed sequence of launches (one persistent work-queue launch does the
 * single-block splitting).  So the call can be captured into a CUDA graph and
 * replayed.  Device-side errors are latched and read by ss_batch_status(). */
ss_status ss_batch_run(ss_batch* b, void* stream);

/* Wait for `stream` and return the device status latched by the last
 * ss_batch_run of this plan. */
ss_status ss_batch_status(ss_batch* b, void* stream);

/* Wait for `stream` and return the device status of the work enqueued on it:
 * first the status word of its ss_sort / ss_sort_ex calls since the last
 * ss_stream_status (which clears it), then that of the last ss_batch_run
 * enqueued on it.  SS_OK if there is neither. */
ss_status ss_stream_status(void* stream);

/* Release a plan (and its workspace if the library allocated it). */
ss_status ss_batch_destroy(ss_batch* b);

/* Convenience: create, run on `stream`, wait, destroy. */
ss_status ss_sort_batch(const ss_set* sets, uint32_t num_sets, const ss_options* opt,
                        void* stream);

/* ---- sorting without allocation -------------------------------------------------- */

#define SS_NOALLOC_MAX_STRINGS 65536u
#define SS_NOALLOC_SCRATCH_BYTES (4u << 20)

/* The paper has no counterpart to this call; it exists for callers that may
 * not allocate device memory while they run (a service that reserves all its
 * GPU memory at start-up, code whose device memory belongs to another
 * allocator, or a latency-critical path on which cudaMalloc / cudaFree, which
 * can synchronise the whole device, are not allowed).
 *
 * Sorts n <= SS_NOALLOC_MAX_STRINGS strings exactly as ss_sort_ex does with
 * default options and this max_len, but calls no cudaMalloc, cudaFree, stream-
 * ordered or pinned allocation: its workspace is a fixed SS_NOALLOC_SCRATCH_BYTES
 * array in the library's device data, which every GPU that loads the library
 * holds until the process exits.  Inputs and outputs are the caller's device
 * buffers, as for ss_sort.  Waits for the sort and returns its status.
 *   - n > SS_NOALLOC_MAX_STRINGS: SS_ERR_TOO_LARGE, nothing is enqueued.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - All calls share the one array and it keeps the last call's contents
 *     (the call clears what must start at zero).  Calls that overlap on the GPU
 *     race with each other: issue them on one stream, or wait for one to end
 *     before the next starts.
 *   - Returns SS_ERR_INVALID while kernel profiling (ss_set_profiling) is on. */
ss_status ss_sort_noalloc(const uint8_t* chars, const uint64_t* offsets, uint64_t n,
                          uint32_t max_len, uint32_t* out_perm, uint32_t* out_lcp, void* stream);

/* ---- diagnostics --------------------------------------------------------------- */

/* Static description of a status code. */
const char* ss_status_string(ss_status s);

/* Number of kernel launches this library has issued in this process: the
 * launches made from the host plus the kernels launched by its multi-block
 * loop graphs on the current device (counted on the device; reading that
 * count waits for the device). */
uint64_t ss_launch_count(void);

/* Per-kernel device timing.  When enabled, the library records CUDA events
 * around each of its kernel launches on the launching stream and accumulates
 * the elapsed time per kernel class once the call has waited for its work
 * (launches of the asynchronous calls ss_merge and ss_distinguishing are
 * waited for and added by the next ss_kernel_stats call of the same thread),
 * together with the algorithmic bytes the kernels of that class moved (the
 * bytes their task requires, counted on the device: each record read and
 * written once, 8 bytes per character-window gather).  ss_kernel_stats fills
 * up to `cap` entries (name, launches, total ms, algorithmic bytes; any output
 * array may be NULL) and returns the number of kernel classes. */
void ss_set_profiling(int enabled);

/* With 0, ss_sort / ss_sort_ex / ss_batch_run run the rounds of multi-block
 * steps from the host instead of the loop graph: the same kernels, each its
 * own launch, with the host waiting for each round's plan (the calls then
 * wait for the multi-block part of the sort).  For tools that cannot see
 * kernels inside a graph with conditional nodes (kernel profilers).  Default
 * 1.  Has no effect on a call made while its stream is being captured. */
void ss_set_graph_loop(int enabled);
uint32_t ss_kernel_stats(const char** names, uint64_t* launches, double* total_ms,
                         uint64_t* alg_bytes, uint32_t cap);
void ss_reset_kernel_stats(void);

#ifdef __cplusplus
}
#endif

#endif /* SS_SORT_H */

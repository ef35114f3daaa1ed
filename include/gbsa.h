/* gbsa — suffix-array construction on one NVIDIA GB300 (sm_103a).
 *
 * Method: prefix doubling with discarding (Bingmann, Gog & Kurpicz,
 * "Scalable Construction of Text Indexes", arXiv 1610.03007, Section 2.1,
 * Algorithms 1, 4 and 5), in inverse-suffix-array form, every step in
 * hand-written CUDA kernels: packed-character initial keys, a one-sweep LSD
 * radix sort with decoupled look-back, boundary flags with a device-wide
 * max-scan for renaming, and stream compaction for discarding.
 *
 * Problem statement (Section 2): for a text T of length n over bytes, the
 * suffix array SA is the permutation of [0,n) with
 * T[SA[i],n) <=lex T[SA[j],n) for i <= j. Bytes compare as unsigned values
 * 0..255 and the end of the text is smaller than every byte (the sentinel $
 * of Section 2.1), so a proper prefix sorts first. Because all suffixes
 * differ, SA is unique; the result is an exact integer permutation.
 *
 * Conventions for every entry point:
 *  - Pointers are DEVICE pointers unless the parameter says HOST.
 *  - All GPU work is ordered on `stream` (a cudaStream_t; NULL = the legacy
 *    default stream). The call returns after the result is complete on the
 *    device: it synchronises `stream` once per doubling round to read the
 *    number of suffixes still active.
 *  - The caller owns every buffer it passes. The library never frees them
 *    and keeps no pointer to them after returning.
 *  - Errors are reported only by the return code; no state is left behind
 *    except that a CUDA error may be sticky in the context (SA_ERR_CUDA).
 *  - Indices and ranks are uint32; n may be at most SA_MAX_N = 2^31.
 *  - Thread safety: calls on different streams with different workspaces
 *    may run concurrently.
 */
#ifndef GBSA_H
#define GBSA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t, declared here so this header needs no CUDA
 * include. */
typedef struct CUstream_st *gbsa_stream_t;

typedef enum {
  SA_OK = 0,
  SA_ERR_INVALID_ARG = 1, /* NULL pointer with n > 0, bad offsets, ...     */
  SA_ERR_TOO_LARGE = 2,   /* n (or the batch total) above SA_MAX_N         */
  SA_ERR_OOM = 3,         /* workspace allocation failed or ws_bytes short */
  SA_ERR_CUDA = 4,        /* a CUDA runtime call or kernel launch failed   */
  SA_ERR_TIMEOUT = 5,     /* a bounded device-side wait (decoupled
                             look-back) expired; the context stays usable  */
  SA_ERR_INTERNAL = 6     /* an internal consistency check failed          */
} sa_status;

#define SA_MAX_N (1ull << 31)
#define SA_MAX_ROUNDS 64

/* Optional knobs for sa_build_ex / sa_build_batched_ex. Zero-initialise and
 * set only what is needed; all-zero means the defaults. */
typedef struct {
  /* Characters packed into the initial 64-bit keys. 0 = as many as fit
   * (floor((64 - segment bits) / bits per character)). A smaller value
   * reproduces the paper's 2-character initial names (Algorithm 1). */
  uint32_t h0_chars;
  /* Maximum polls of one decoupled look-back wait before the kernel gives
   * up with SA_ERR_TIMEOUT. 0 = default (about one second). */
  uint32_t spin_limit;
  /* Test hook: when 1, the first tile of the first radix pass never
   * publishes its counts, so the next tile's bounded wait must expire and
   * the call must return SA_ERR_TIMEOUT. 0 in normal use. */
  uint32_t inject_stall;
  /* If not NULL: DEVICE buffer of trace_cap * n uint32. The name (ISA
   * value) of every position after the initial naming and after each
   * refinement round k is written to trace_isa[k*n .. k*n+n) for
   * k < trace_cap (single text only). */
  uint32_t *trace_isa;
  uint32_t trace_cap;
  /* Group names between rounds. 0 (default): a split group's name stays
   * with the subgroup whose SA interval contains it and every other
   * subgroup takes the middle of its interval, so a majority subgroup keeps
   * its name and fewer ISA entries are rewritten. 1: the paper's names, the
   * start of the interval (Algorithms 5/6, NameDiscarding), so that the
   * per-round names in trace_isa equal the paper's. Both give the same SA
   * and ISA; any rank inside a group's interval is a valid lexicographic
   * name (Section 2). */
  uint32_t paper_names;
  /* Tile shape of the small-group refine of rounds >= 1 (threads per block
   * x items per tile): 0 = automatic, 1 = 128 x 1024, 2 = 256 x 2048,
   * 3 = 256 x 4096, 4 = 256 x 1024. Groups of up to half a tile are refined
   * inside one tile; larger ones take the global radix sort. Any other
   * value: SA_ERR_INVALID_ARG. */
  uint32_t refine_shape;
  /* Keys per thread of the one-sweep radix pass (tile = 256 x this):
   * 8, 12 or 16; 0 = automatic (16). Any other value: SA_ERR_INVALID_ARG. */
  uint32_t sort_items;
  /* When 1, CUDA events are recorded on `stream` around every kernel launch
   * and the per-kernel-class times, launch counts and algorithmic bytes are
   * returned in sa_stats (adds a few microseconds per launch). */
  uint32_t profile;
  /* Growth factor a of the resolved prefix per round (Section 2.1, Prefix
   * Quadrupling: substrings of length a^k instead of 2^k). Each round ranks
   * the names of i, i + h, ..., i + (a-1)h, so h grows a-fold and fewer
   * rounds run; 0 or 2 = doubling (default), 3 = tripling, 4 =
   * quadrupling. Any other value: SA_ERR_INVALID_ARG. The SA and ISA are
   * the same for every a; trace_isa holds the names after each round, at
   * h0 * a^k resolved characters. */
  uint32_t multiplier;
  /* Discard threshold: when at least this many ISA writes may be pending
   * (names of suffixes discarded as unique, or renamed, in a round; Section
   * 2.1, Algorithms 5 and 6), they are first bucketed by position so that
   * the writes stay in L2; fewer are written directly. 0 = automatic (the
   * tuning table, else 2^22); 0xFFFFFFFF = never bucket. Same SA and ISA
   * for every value. */
  uint32_t bucket_min;
  /* Rounds after round 0 without a host round trip per round (Algorithm 5's
   * loop on the GPU): they run as one CUDA graph, a while-node whose body
   * is two rounds of persistent kernels that read their sizes from a device
   * round state, with if-nodes for the optional steps. 0 = the library
   * chooses, 1 = device-driven, 2 = host-driven (one 64-byte readback and
   * stream synchronisation per round). Doubling only: with multiplier 3 or
   * 4, a name trace or profile = 1 the rounds are host-driven. Same SA and
   * ISA either way. */
  uint32_t device_rounds;
  /* Order of the groups of equal names in the active list after round 0:
   * 0 = the library chooses (the position order below whenever a round
   * follows), 1 = ordered by each group's smallest member position, so that
   * groups of suffixes that move together (copies of a repeated text) sit
   * side by side and their partner-name reads share cache lines, 2 = rank
   * order (as round 0 leaves them). Same SA and ISA either way: a round
   * needs each group contiguous, not in any order (names are ranks). */
  uint32_t group_order;
  /* Where round 0's initial keys (Algorithm 1's initial names, c0
   * characters each) are formed: 0 = the library chooses (as 1 whenever it
   * applies), 1 = inside the first radix pass, which reads the text and
   * writes the keys once sorted by their lowest digit, so no packed copy is
   * written and read back (one text whose digits hold whole characters:
   * 1, 2, 4 or 8 bits per character and c0 * bits a multiple of 8; else as
   * 2), 2 = by a separate pass that writes every key and position first.
   * Any other value: SA_ERR_INVALID_ARG. Same SA and ISA either way. */
  uint32_t initial_keys;
} sa_options;

/* Tuned build parameters (the autotuner's table, see sa_tuning_set): each
 * field as the sa_options field of the same name; 0 = built-in default. */
typedef struct {
  uint32_t sort_items;
  uint32_t refine_shape;
  uint32_t h0_chars;
  uint32_t bucket_min;
} sa_tuned;

/* Kernel classes of the per-kernel statistics. */
enum {
  SA_K_BYTE_HIST = 0, /* alphabet histogram                  */
  SA_K_PACK = 1,      /* initial packed keys                 */
  SA_K_DIGIT_HIST = 2,/* radix digit histograms              */
  SA_K_PLAN = 3,      /* radix plan (one block)              */
  SA_K_ONESWEEP = 4,  /* radix passes (kept passes only)     */
  SA_K_RENAME = 5,    /* rename + unique + compaction        */
  SA_K_GATHER = 6,    /* partner-name gather (large groups)  */
  SA_K_OUTPUT = 7,    /* output fix-ups                      */
  SA_K_REFINE = 8,    /* small-group refine (rounds >= 1)    */
  SA_K_SCATTER = 9,   /* deferred ISA updates                */
  SA_K_CLASSIFY = 10, /* group classification, tile map      */
  SA_K_APPLY = 11,    /* ISA entries of renamed survivors    */
  SA_K_BUCKET = 12,   /* position bucketing of ISA writes    */
  SA_K_REORDER = 13,  /* group order after round 0           */
  SA_K_CLASSES = 14
};

/* Per-build statistics (HOST struct filled by the _ex calls). */
typedef struct {
  uint32_t rounds;          /* doubling rounds including round 0          */
  uint32_t sigma;           /* distinct byte values in the input          */
  uint32_t bits_per_char;   /* b = ceil(log2 sigma), at least 1           */
  uint32_t chars_per_key;   /* c0: characters in the initial keys         */
  uint64_t active[SA_MAX_ROUNDS];  /* m_r: suffixes sorted in round r     */
  uint64_t unique[SA_MAX_ROUNDS];  /* u_r: suffixes that became unique    */
  uint32_t passes[SA_MAX_ROUNDS];  /* radix passes executed in round r    */
  uint32_t key_bits[SA_MAX_ROUNDS];/* significant key bits in round r     */
  uint64_t groups[SA_MAX_ROUNDS];  /* groups of equal names left after r  */
  /* Algorithmic bytes moved (reads + writes, 4 bytes per random access)
   * summed over all kernels and rounds; the model is documented with the
   * kernels. */
  uint64_t bytes_model;
  /* Kernel launches issued by the build (all classes, skipped radix passes
   * included). */
  uint32_t launches;
  /* With sa_options.profile = 1, per kernel class (SA_K_*): summed
   * event-timed milliseconds, launches timed, and algorithmic bytes. */
  double kernel_ms[SA_K_CLASSES];
  uint64_t kernel_launches[SA_K_CLASSES];
  uint64_t kernel_bytes[SA_K_CLASSES];
  /* The parameters the build ran with (its options, else the tuning table's
   * entry for its class, else the defaults): radix keys per thread, refine
   * tile shape (1-4), discard threshold; chars_per_key above is the key
   * width. tuned = 1 when at least one came from the tuning table. */
  uint32_t sort_items, refine_shape, bucket_min, tuned;
} sa_stats;

/* Suffix array of one text (Section 2; Algorithm 5).
 * text   : DEVICE, n bytes, read only.
 * n      : length, 0 <= n <= SA_MAX_N.
 * sa_out : DEVICE, n uint32, written with SA.
 * The workspace (about 67 bytes per character plus 1 MiB) is allocated from a
 * library-private stream-ordered pool on `stream` and returned to it.
 * n = 0 writes nothing; n = 1 writes sa_out[0] = 0. */
sa_status sa_build(const uint8_t *text, uint64_t n, uint32_t *sa_out,
                   gbsa_stream_t stream);

/* Workspace size sa_build_ex needs for a text of n bytes. */
size_t sa_workspace_bytes(uint64_t n);

/* sa_build with an optional ISA output, a caller-owned workspace, options
 * and statistics.
 * isa_out   : DEVICE, n uint32 or NULL; receives ISA (ISA[SA[j]] = j).
 * workspace : DEVICE, ws_bytes >= sa_workspace_bytes(n), 256-byte aligned,
 *             or NULL to allocate internally. Contents need no
 *             initialisation and are garbage afterwards.
 * opt, stats: HOST, either may be NULL. */
sa_status sa_build_ex(const uint8_t *text, uint64_t n, uint32_t *sa_out,
                      uint32_t *isa_out, void *workspace, size_t ws_bytes,
                      const sa_options *opt, sa_stats *stats,
                      gbsa_stream_t stream);

/* Suffix arrays of `count` independent texts in one launch sequence.
 * texts   : DEVICE, the texts concatenated, offsets[count] bytes.
 * offsets : HOST, count+1 uint64, offsets[0] = 0, non-decreasing; text k is
 *           texts[offsets[k] .. offsets[k+1]). Empty texts are allowed.
 * sa_out  : DEVICE, offsets[count] uint32. The SA of text k is written to
 *           sa_out[offsets[k] .. offsets[k+1]) with LOCAL indices
 *           (0 .. len_k - 1).
 * Every text has its own end sentinel; texts never compare with each other.
 * offsets[count] may be at most SA_MAX_N and count at most 2^20. */
sa_status sa_build_batched(const uint8_t *texts, const uint64_t *offsets,
                           uint32_t count, uint32_t *sa_out,
                           gbsa_stream_t stream);

/* Workspace size sa_build_batched_ex needs. offsets: HOST, count+1. */
size_t sa_batched_workspace_bytes(const uint64_t *offsets, uint32_t count);

/* sa_build_batched with a caller-owned workspace, options and statistics
 * (same rules as sa_build_ex; trace_isa is ignored). */
sa_status sa_build_batched_ex(const uint8_t *texts, const uint64_t *offsets,
                              uint32_t count, uint32_t *sa_out, void *workspace,
                              size_t ws_bytes, const sa_options *opt,
                              sa_stats *stats, gbsa_stream_t stream);

/* End-to-end build from HOST memory: copies host_text (HOST, n bytes) to the
 * device on `stream`, builds, and copies SA back to host_sa (HOST, n
 * uint32). Pinned host buffers give the fastest copies; pageable buffers
 * work. With both buffers pinned and n <= 4 MiB the copies run as kernels
 * through the buffers' device mapping instead of on a copy engine, where
 * they would wait behind the large copies of builds on other streams.
 * Device memory (text, SA and workspace) comes from the library pool. */
sa_status sa_build_host(const uint8_t *host_text, uint64_t n, uint32_t *host_sa,
                        gbsa_stream_t stream);

/* sa_build_host for `count` texts at once, built together as one batch
 * (sa_build_batched: shared doubling rounds, each text leaving them as soon
 * as all its suffixes are unique), the form the server uses to merge the
 * small requests queued at one moment into one build.
 * host_texts : HOST array of count HOST pointers; text k has lengths[k]
 *              bytes (its pointer may be NULL when lengths[k] = 0).
 * lengths    : HOST, count uint64.
 * host_sas   : HOST array of count HOST pointers; host_sas[k] receives the
 *              SA of text k (lengths[k] uint32, local indices).
 * The texts are gathered into one device buffer and the SAs scattered
 * back: when the total is at most 4 MiB and every buffer is pinned, by one
 * kernel launch per 64 texts in each direction (through the buffers'
 * device mapping); otherwise one copy-engine copy per text and direction.
 * Device memory comes from the library pool; returns after the stream has
 * synchronised. SA_ERR_INVALID_ARG for count = 0 or a NULL array or
 * non-empty text's pointer; SA_ERR_TOO_LARGE for count > 2^20 or a total
 * above SA_MAX_N. Each SA is exactly sa_build's for that text. */
sa_status sa_build_batched_host(const uint8_t *const *host_texts, const uint64_t *lengths,
                                uint32_t *const *host_sas, uint32_t count,
                                gbsa_stream_t stream);

/* Stable LSD radix sort of (key, value) pairs by key bits
 * [begin_bit, end_bit), the building block of the sort step (Algorithm 1,
 * "Sort triples by name pair"). One-sweep passes of 8-bit digits with
 * decoupled look-back; digits that are equal for all keys are skipped.
 * keys, vals : DEVICE, m entries each; sorted in place (the library copies
 *              back if the result lands in the workspace buffers).
 * workspace  : DEVICE, >= sa_sort_workspace_bytes(m), or NULL (pool).
 * 0 <= begin_bit < end_bit <= 64, m <= SA_MAX_N. */
sa_status sa_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t m,
                        uint32_t begin_bit, uint32_t end_bit, void *workspace,
                        size_t ws_bytes, gbsa_stream_t stream);
size_t sa_sort_workspace_bytes(uint64_t m);

/* ---- The autotuner's table ---------------------------------------------
 * Build parameters picked by measurement (radix tile, refine tile shape,
 * initial key width, discard threshold) per workload class: single text or
 * batch (batched 0 or 1), bits per character of the alphabet (1..8, as the
 * build computes it from the byte histogram), floor(log2) of the total
 * length (0..31). A build whose sa_options leave a knob at 0 takes it from
 * the entry of its own (batched, bits) class with the nearest size, else
 * the built-in default; sa_stats reports what it ran with. The table is
 * read at the first lookup from the file named by GBSA_TUNING_TABLE, else
 * tuning.txt beside libgbsa.so (written by autotune.py), one entry a line:
 * "batched bits log2n sort_items refine_shape h0_chars bucket_min".
 * The paper has no counterpart: this chooses how the library runs the sort
 * and discard steps of Section 2.1, not what they compute. Thread-safe;
 * allocates no device memory. */

/* Sets (params non-NULL, HOST) or removes (NULL) one entry. Returns
 * SA_ERR_INVALID_ARG for a key out of range. */
sa_status sa_tuning_set(uint32_t batched, uint32_t bits_per_char, uint32_t log2_n,
                        const sa_tuned *params);
/* Replaces the whole table by the file at path (NULL: an empty table).
 * SA_ERR_INVALID_ARG if the file cannot be read or a line is malformed
 * (the table is left unchanged then). */
sa_status sa_tuning_load(const char *path);
/* The parameters a build of this class and total length n would take from
 * the table (all 0 if none applies) into *out (HOST); returns the number of
 * entries in the table. */
uint32_t sa_tuning_lookup(uint32_t batched, uint32_t bits_per_char, uint64_t n, sa_tuned *out);

/* Device memory held by the library's own stream-ordered pool on the
 * current device, which sa_build, sa_build_batched, sa_build_host,
 * sa_sort_pairs (without a caller workspace) and the DC3/DC7 and sorting
 * variants draw from: *used = bytes handed out now, *reserved = bytes the
 * pool holds from the device (it is never trimmed). Both 0 before the first
 * allocation on this device. used, reserved: HOST. Returns
 * SA_ERR_INVALID_ARG for a NULL pointer, SA_ERR_CUDA if the device cannot
 * be queried. Allocates nothing; the paper has no counterpart (a runtime
 * query). */
sa_status sa_pool_usage(uint64_t *used, uint64_t *reserved);

/* Returns the current device's pool memory that no build holds to the
 * device, keeping at most keep_bytes reserved (cudaMemPoolTrimTo). Memory
 * of builds still in flight is not touched; call it after they completed
 * (synchronise their streams first) to hand the memory to other users.
 * SA_ERR_CUDA if the device cannot be queried. The paper has no
 * counterpart (a runtime call). */
sa_status sa_pool_trim(uint64_t keep_bytes);

/* sa_build without any device memory allocation, for callers that must not
 * allocate when they build: for example code running beside a serving
 * engine or framework allocator that already reserved the GPU's memory, a
 * latency-sensitive path that cannot afford cudaMalloc's implicit
 * synchronisation, or a plug-in whose host forbids device allocation.
 * The paper has no counterpart; this is a packaging of the same build.
 * text, n, sa_out, stream: as for sa_build. n may be at most 2^18
 * (262144); larger n returns SA_ERR_TOO_LARGE.
 * The workspace is a 20 MiB array in the library's own device memory, held
 * on every GPU that loads the library until the process exits. Each call
 * looks up that array's device address in the current context (a CUDA
 * runtime query that allocates nothing). Like sa_build, a call synchronises
 * `stream` once per doubling round, so it cannot be made while that stream
 * is being captured into a CUDA graph. All calls share the one array: calls
 * whose GPU work overlaps race and give garbage, so serialise them (one
 * stream, or an event between streams). Leftover contents from the
 * previous call are harmless: every build clears what it needs. */
sa_status sa_build_noalloc(const uint8_t *text, uint64_t n, uint32_t *sa_out,
                           gbsa_stream_t stream);

/* ---- Serving: continuous batching of SA builds --------------------------
 * A server owns `slots` worker threads, each with its own CUDA stream.
 * Requests (a HOST text and a HOST output buffer) queue in arrival order;
 * the request at the head of the queue starts as soon as a slot is free
 * and its device footprint (sa_request_footprint) fits in what is left of
 * `budget_bytes`. Each running request keeps its text, SA and workspace
 * (rank and ISA state) resident on the device for all its rounds and frees
 * them when it completes, so requests that arrive while others run are
 * admitted as slots and memory free up, and the builds in flight overlap
 * on the device. With merge_requests >= 2, a worker that takes a small
 * request also takes the small requests queued directly behind it and
 * builds them as one batch (sa_build_batched_host): one launch sequence and one set of doubling
 * rounds for all of them, each text leaving the rounds once its suffixes
 * are unique. Every request's result is exactly sa_build's. */
typedef struct sa_server sa_server;

typedef struct {
  uint64_t budget_bytes;      /* device bytes in use at once; 0 = 100 GB        */
  uint32_t slots;             /* builds in flight at once; 0 = 8, at most 64    */
  int32_t device;             /* CUDA device of the workers (-1 = current)      */
  /* Test hook: when non-zero no GPU work is done; a request "runs" for
   * n * simulate_ns_per_byte nanoseconds and its SA buffer is untouched. */
  uint32_t simulate;
  double simulate_ns_per_byte;
  /* 0 (default): a request runs on a CUDA stream whose priority falls with
   * its size (up to 256 KiB the device's highest priority, then one level
   * lower for each size class up to 2 MiB, 16 MiB and beyond), so the
   * block scheduler starts a small request's blocks before the waiting
   * blocks of large builds in flight and its latency stays near that of a
   * build alone. 1: every request on a stream of default priority. */
  uint32_t size_priority;
  /* Most requests one build takes: a worker that takes a request of at
   * most 256 KiB also takes the requests queued directly behind it while
   * each is at most 256 KiB, the batch stays within 4 MiB of text, its
   * footprint (text, SA and batched workspace) fits in the budget and it
   * holds no more than the worker's share of the queue (the queued requests
   * divided among the idle workers, this one included, rounded up), so
   * requests merge only when the queue outgrows the idle workers. The batch
   * is built by sa_build_batched_host. Queue order is kept. 0 (default)
   * or 1 = every request built alone; values above 64 mean 64. */
  uint32_t merge_requests;
} sa_server_config;

typedef struct {
  sa_status status;           /* result of the build (SA_OK when done well)     */
  uint64_t n;                 /* text length                                     */
  uint32_t slot;              /* worker that ran it                              */
  double submit_s, start_s, done_s; /* seconds since the server was created     */
  int32_t priority;           /* CUDA stream priority it ran at (lower = higher; */
                              /* in simulate mode the range [-5, 0] is assumed) */
  uint32_t batch;             /* requests in the build it ran in (1 = alone)     */
} sa_request_info;

typedef struct {
  uint64_t submitted, completed;
  uint64_t bytes_in_use, peak_bytes_in_use;
  uint32_t in_flight, peak_in_flight, queued;  /* requests (not builds)      */
  uint32_t tracked;           /* requests held: queued, running or uncollected */
  uint64_t builds;            /* builds started (a merged batch counts once)   */
  uint64_t merged;            /* requests that ran in a batch of two or more   */
} sa_server_stats;

/* Device bytes a request of n characters holds while it runs (text, SA and
 * build workspace). */
size_t sa_request_footprint(uint64_t n);

/* Creates a server (cfg HOST, may be NULL for the defaults). */
sa_status sa_server_create(const sa_server_config *cfg, sa_server **out);

/* Queues a request. host_text (n bytes) and host_sa (n uint32) are HOST
 * buffers owned by the caller that must stay valid until the request is
 * done. *ticket identifies it. A request whose footprint exceeds the whole
 * budget is refused with SA_ERR_OOM; n > SA_MAX_N with SA_ERR_TOO_LARGE. */
sa_status sa_server_submit(sa_server *s, const uint8_t *host_text, uint64_t n,
                           uint32_t *host_sa, uint64_t *ticket);

/* 1 if the request is done (info filled), 0 if pending, -1 if the ticket
 * is unknown. Non-blocking. Reporting 1 hands the result over: the server
 * forgets the request and its ticket becomes unknown. */
int sa_server_poll(sa_server *s, uint64_t ticket, sa_request_info *info);

/* Blocks until the request is done; returns its status (info may be NULL).
 * On return the server has forgotten the request (its ticket is unknown to
 * later calls; several threads may wait on one ticket at once). An unknown
 * ticket gives SA_ERR_INVALID_ARG. */
sa_status sa_server_wait(sa_server *s, uint64_t ticket, sa_request_info *info);

/* Current counters (HOST struct). */
void sa_server_get_stats(sa_server *s, sa_server_stats *out);

/* Finishes every queued and running request, stops the workers and frees
 * the server. */
void sa_server_destroy(sa_server *s);

/* ---- Burrows-Wheeler transform from the suffix array ------------------
 * The direct consumer of SA named as future work at the end of the paper
 * (Section 3, the Conclusion); BWT[r] = T[SA[r] - 1] by the definitions of Section 2.
 * Rows are those of T$ (n + 1): row 0 is the suffix $ alone, preceded by
 * T[n - 1]; row r >= 1 is the suffix sa[r - 1], preceded by
 * T[sa[r - 1] - 1], except the row whose suffix is T itself, which holds $
 * stored as byte 0; its row index is the primary index.
 * text        : DEVICE, n bytes, read only.
 * sa          : DEVICE, n uint32, the suffix array of text (sa_build).
 * bwt_out     : DEVICE, n + 1 bytes, written.
 * primary_out : DEVICE, one uint64, written with the primary index
 *               (0 for n = 0).
 * Stream-ordered on `stream`; allocates nothing. Returns SA_ERR_INVALID_ARG
 * for a NULL pointer (text and sa may be NULL when n = 0) and
 * SA_ERR_TOO_LARGE for n > SA_MAX_N. An sa that is not a suffix array of
 * text gives an unspecified BWT but no out-of-bounds access. */
sa_status sa_bwt(const uint8_t *text, uint64_t n, const uint32_t *sa, uint8_t *bwt_out,
                 uint64_t *primary_out, gbsa_stream_t stream);

/* ---- LCP array from the suffix array -----------------------------------
 * The other direct consumer of SA named as future work (Section 3):
 * lcp_out[0] = 0 and, for j >= 1, lcp_out[j] = the length of the longest
 * common prefix of the suffixes sa[j-1] and sa[j] (Section 2's order).
 * Computed in the permuted form of Kasai et al.'s algorithm (Phi, PLCP).
 * text      : DEVICE, n bytes, read only.
 * sa        : DEVICE, n uint32, the suffix array of text (sa_build).
 * lcp_out   : DEVICE, n uint32, written.
 * workspace : DEVICE, ws_bytes >= sa_lcp_workspace_bytes(n) (about 20 bytes
 *             per character plus 1 MiB: Phi, PLCP and, from 2^20
 *             characters on, the Phi writes grouped by position), 256-byte
 *             aligned; NULL to have it allocated and freed stream-ordered
 *             on `stream` (cudaMallocAsync).
 * Stream-ordered on `stream`. Returns SA_ERR_INVALID_ARG for a NULL text,
 * sa or lcp_out with n > 0, or a short or misaligned workspace;
 * SA_ERR_TOO_LARGE for n > SA_MAX_N; SA_ERR_OOM if the allocation fails.
 * An sa that is not a suffix array of text gives unspecified values but no
 * out-of-bounds access. n = 0 writes nothing. */
size_t sa_lcp_workspace_bytes(uint64_t n);
sa_status sa_lcp(const uint8_t *text, uint64_t n, const uint32_t *sa, uint32_t *lcp_out,
                 void *workspace, size_t ws_bytes, gbsa_stream_t stream);

/* ---- DC3 (difference cover modulo 3) -----------------------------------
 * The suffix array by the skew algorithm (Karkkainen and Sanders; the
 * paper's Section 2.2, Algorithm 7, gives its distributed form): the
 * suffixes at positions i mod 3 != 0 are ranked by recursion on the string
 * of their triples' names, those at i mod 3 = 0 are sorted by (T[i], rank
 * of i + 1), and the two are merged. Same result as sa_build.
 * text        : DEVICE, n bytes, read only.
 * sa_out      : DEVICE, n uint32, written with SA.
 * trace_names : DEVICE or NULL; if set, n0 + n2 uint32 (n0 = (n+2)/3,
 *               n2 = n/3) are written: the top level's recursion string,
 *               the 1-based names of the triples at positions 1 mod 3
 *               (with the position n itself when n mod 3 = 1), then at
 *               positions 2 mod 3.
 * Memory comes from the library's stream-ordered pool; the call
 * synchronises `stream` once per recursion level and before returning.
 * Returns SA_ERR_INVALID_ARG for a NULL text or sa_out with n > 0,
 * SA_ERR_TOO_LARGE for n > SA_MAX_N, SA_ERR_OOM if memory runs out.
 * n = 0 writes nothing. */
sa_status sa_build_dc3(const uint8_t *text, uint64_t n, uint32_t *sa_out, uint32_t *trace_names,
                       gbsa_stream_t stream);

/* ---- DC7 (difference cover modulo 7) -----------------------------------
 * The suffix array by DC7 (Section 2.2, Algorithms 8-10): the suffixes at
 * the positions of the difference cover D7 = {0, 1, 3} modulo 7 are ranked
 * by recursion on the string of the names of their 7-character windows;
 * every position's suffix is then placed within its class i mod 7 by at
 * most three characters and one sample's rank, and the seven classes are
 * merged, two suffixes comparing by their first l characters and the ranks
 * l positions on, l the smallest offset taking both into D7. Same result
 * as sa_build.
 * text        : DEVICE, n bytes, read only.
 * sa_out      : DEVICE, n uint32, written with SA.
 * trace_names : DEVICE or NULL; if set, m = c0 + c1 + c3 uint32 are
 *               written, c_a = floor((n - a) / 7) + 1 for a <= n (else 0):
 *               the top level's recursion string, the 1-based names of the
 *               7-character windows of the positions i = 0 mod 7 with
 *               i <= n in text order, then of i = 1 mod 7, then of
 *               i = 3 mod 7 (3 * (n / 7 + 1) entries always suffice).
 * Memory (about 100 bytes per character at the top level) comes from the
 * library's stream-ordered pool; the call synchronises `stream` twice per
 * recursion level and before returning. Returns SA_ERR_INVALID_ARG for a
 * NULL text or sa_out with n > 0, SA_ERR_TOO_LARGE for n > SA_MAX_N,
 * SA_ERR_OOM if memory runs out. n = 0 writes nothing. */
sa_status sa_build_dc7(const uint8_t *text, uint64_t n, uint32_t *sa_out, uint32_t *trace_names,
                       gbsa_stream_t stream);

/* ---- Prefix doubling using sorting -------------------------------------
 * The suffix array by prefix doubling without discarding, with the partner
 * names fetched by sorting instead of through the inverse suffix array
 * (Section 2.1, Algorithms 1, 2 and 3): every round sorts all n suffixes
 * by their name pair, names them by CmpName and PrefixSum(max) (head
 * ranks), and unless all names differ sorts the (position, name) items by
 * the comparator of Eq. 1, (i mod 2^k, i div 2^k), so that each name's
 * partner i + 2^k is its successor. The initial names are the character
 * pairs (T[i], T[i+1]) with T[n] = $. Same result as sa_build.
 * text        : DEVICE, n bytes, read only.
 * sa_out      : DEVICE, n uint32, written with SA.
 * trace_names : DEVICE or NULL; if set, trace_cap * n uint32: row r holds
 *               every position's name after the r-th naming (row 0: the
 *               character pairs), for r < trace_cap.
 * rounds      : HOST or NULL; receives the number of namings.
 * Memory comes from the library's stream-ordered pool; the call
 * synchronises `stream` once per round and before returning. Returns
 * SA_ERR_INVALID_ARG for a NULL text or sa_out with n > 0,
 * SA_ERR_TOO_LARGE for n > SA_MAX_N, SA_ERR_OOM if memory runs out.
 * n = 0 writes nothing. */
sa_status sa_build_pd_sort(const uint8_t *text, uint64_t n, uint32_t *sa_out,
                           uint32_t *trace_names, uint32_t trace_cap, uint32_t *rounds,
                           gbsa_stream_t stream);

/* Human-readable name of a status code (static string). */
const char *sa_status_string(sa_status s);

#ifdef __cplusplus
}
#endif
#endif

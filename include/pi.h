/*
 * pi.h -- C ABI of the GB300 (sm_103a) implementation of PI's batch hot path.
 *
 * PI ("a Parallel in-memory skip list based Index", arXiv:1601.00159) keeps a
 * sorted storage layer of data nodes (key, value, height, delete flag; Definition 1
 * and Section 3.2.3) under an index layer of sorted levels (Section 3.1). It answers
 * a whole batch of point queries at once (Algorithm 1): sort the batch by key,
 * descend the index layer to each query's interception (Algorithm 2, Definition 4),
 * give every storage node a single owner (Algorithm 3 and Section 3.2.4), execute
 * the queries against the storage layer (Algorithm 4), and rebuild the index layer
 * from the storage layer (Sections 4.1 and 4.4.4).
 *
 * All array arguments are DEVICE pointers unless a name ends in _host. They are owned
 * by the caller and must stay valid until the work that reads them has completed on
 * the stream passed in. Keys and values are unsigned 64-bit integers compared as
 * unsigned; the key 2^64-1 is reserved (it is the sentinel that ends every level).
 *
 * Threading: a pi_index_t must not be used from two host threads at the same time. Its
 * calls may name different streams: every call that touches the index is ordered, on
 * the device, after the index's previous operation (a batch, a range search or a
 * batching-form call), whichever stream that ran on.
 */
#ifndef PI_H_
#define PI_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ABI-identical to cudaStream_t; NULL means the legacy default stream. */
typedef struct CUstream_st* pi_stream_t;

typedef struct pi_index pi_index_t; /* opaque, library-owned device state */

/* One result per query, in arrival order (16 bytes). */
typedef struct {
    uint64_t value;    /* the key's value just before this query, or 0 if it was absent */
    uint32_t status;   /* PI_R_* */
    uint32_t reserved; /* always 0 */
} pi_result_t;

/* Query types (Definition 2: a query is (type, key, [value])). */
enum { PI_OP_SEARCH = 0, PI_OP_INSERT = 1, PI_OP_DELETE = 2 };

/* Per-query status. */
enum {
    PI_R_ABSENT = 0,  /* the key was not present before this query */
    PI_R_PRESENT = 1, /* the key was present; value holds its value */
    PI_R_INVALID = 2  /* op code not 0/1/2, or key == 2^64-1: the query had no effect */
};

/* Return codes. */
enum {
    PI_OK = 0,
    PI_ERR_INVALID_ARG = -1, /* NULL pointer, size over a limit, bad promote_p, reserved key */
    PI_ERR_OOM = -2,         /* device allocation failed; the index is unchanged */
    PI_ERR_CUDA = -3,        /* a CUDA call failed (launch error or an earlier fault) */
    PI_ERR_TIMEOUT = -4,     /* a bounded device-side wait gave up; the index is unusable */
    PI_ERR_NOT_BUILT = -5    /* pi_export_level: that level is not materialised */
};

#define PI_MAX_BATCH (1u << 28)          /* queries per pi_execute_batch call */
#define PI_MAX_KEYS ((1u << 30) - 2u)    /* storage-layer nodes */

/* Optional tuning for pi_create_ex. Zero means "default" for every field. */
typedef struct {
    uint32_t struct_size;        /* sizeof(pi_config_t) */
    uint32_t rebuild_policy;     /* 0: rebuild the index layer after every batch that
                                    changed it (default). 1: deferred, as in Section 6's
                                    setup: rebuild only when the storage layer was
                                    re-laid-out or the updates since the last rebuild
                                    exceed rebuild_threshold_pct percent of its size. */
    uint32_t rebuild_threshold_pct; /* policy 1 only; default 15 (Section 6) */
    uint32_t smem_top_entries;   /* cap on the index entries staged in shared memory by the
                                    descent (default and maximum 12288); smaller values
                                    pin fewer top levels */
    uint64_t storage_capacity;   /* initial storage-layer capacity, in nodes */
    uint64_t index_capacity;     /* initial index-layer capacity, in entries */
    uint32_t test_flags;         /* PI_TEST_*: alternative code paths for tests; 0 in use */
    uint32_t lowest_level;       /* lowest index level to materialise, 2..16. 0: automatic,
                                    the lowest level l whose expected storage gap (1/P)^(l-1)
                                    is at least 32 nodes (4 for P = 1/4), since on the GPU the
                                    storage search interpolates within a gap and reads about
                                    one 64-byte line of it, while every built level costs a
                                    rebuild pass and a descent step. 2 builds every level, as
                                    the paper does. Levels below it still count in
                                    pi_info's level sizes; pi_export_level reports them as
                                    PI_ERR_NOT_BUILT. */
    uint32_t sort_passes;        /* radix passes per batch. 0: automatic, four on the most
                                    significant key bytes that vary in the batch, then an
                                    ordering of the queries whose keys agree on those bytes
                                    (all eight for the next batches while such queries
                                    exceed 1/16 of a batch). 1..4: that many passes on the
                                    most significant varying bytes, then that ordering.
                                    8: every varying byte. Every choice gives the same
                                    results. (Callers built against the header without this
                                    field pass a smaller struct_size; it then reads as 0.) */
    uint32_t small_batches;      /* 0: every batch takes the level-synchronous pipeline
                                    (default). 1: a batch of at most 2^16 queries on an
                                    index of at most 2^20 nodes (its new keys included)
                                    runs as one launch, the batching form's pipeline on a
                                    thread-block cluster of 16 CTAs of 16 warps (8 where 16
                                    do not fit), with the same results. Measured on a
                                    GB300 it is about as fast as the default for such
                                    batches (98 against 99 us for 2^14 searches on 2^16
                                    keys; faster on the smallest batches, slower on 2^12
                                    queries on 2^18 keys). Not taken while profiling, with
                                    test_flags or with the deferred rebuild policy. */
} pi_config_t;

/* test_flags bit: give only the lowest index level a launch of its own in the
 * level-synchronous descent, so every other level takes the in-kernel walk. */
#define PI_TEST_WALK_LEVELS 1u
/* test_flags bit: sort every batch with all eight radix passes (no prefix fix-up). */
#define PI_TEST_SORT_FULL 2u
/* test_flags field (bits 4-6): sort batches with only k = 1..4 radix passes on the most
 * significant varying key bytes, so the fix-up that orders key-prefix segments sees
 * many long segments. The default is four passes. */
#define PI_TEST_SORT_PREFIX(k) ((uint32_t)(k) << 4)
/* test_flags bit: debug check of single ownership (Section 3.2.4). Each batch counts the
 * writes to every storage node (4 B per node of capacity); a node written twice records
 * a sticky error (pi_status then returns PI_ERR_CUDA), and pi_info's
 * owner_checked_writes sums the writes checked. The batching form is not checked. */
#define PI_TEST_OWNER_CHECK 0x100u

/*
 * pi_create -- bulk-build an index from n (key, value) pairs (Section 3.1: the index
 * layer is built bottom-up by one scan of the storage layer).
 *   keys, values: device arrays of n entries. A key that appears several times keeps
 *     its LAST value, as if the pairs were inserted in order.
 *   promote_p: the promotion probability P of Definition 1; must be 1/2, 1/4, 1/8 or
 *     1/16. A key's tower height is 1 + min(ctz(h) / b, Hmax - 1) with p = 2^-b,
 *     h = splitmix64(key ^ splitmix64(seed)), Hmax = min(32, 64 / b), ctz(0) = 64.
 *   seed: seeds the height hash; the structure is a pure function of keys and seed.
 * Synchronous. Returns NULL on error; pi_last_error() then gives the code
 * (PI_ERR_INVALID_ARG for n > PI_MAX_KEYS, a bad promote_p or a reserved key).
 */
pi_index_t* pi_create(const uint64_t* keys, const uint64_t* values, uint64_t n,
                      double promote_p, uint64_t seed);
pi_index_t* pi_create_ex(const uint64_t* keys, const uint64_t* values, uint64_t n,
                         double promote_p, uint64_t seed, const pi_config_t* config);

/*
 * pi_execute_batch -- process one query set Q (Definition 3; Algorithm 1).
 *   ops[n] (uint8), keys[n], values[n] (values read only where ops[i] == PI_OP_INSERT),
 *   results[n]: device arrays. Results are in arrival order: query i reports the
 *   state of its key just before query i, as if the batch were applied one query at
 *   a time in arrival order (the batch is serializable, Section 4.2). Insert sets the
 *   key's value and clears its delete flag (Algorithm 4); delete sets the flag; search
 *   changes nothing. For a search this is Algorithm 4's result; for a delete PRESENT
 *   is the paper's "return 1"; for an insert the paper returns null and this library
 *   reports the prior state instead.
 * Stream-ordered and asynchronous: results are complete when `stream` completes.
 * No host synchronisation happens except, rarely, when a capacity must grow.
 * n == 0 is a no-op. Returns PI_ERR_INVALID_ARG for NULL pointers or n > PI_MAX_BATCH,
 * PI_ERR_OOM if a capacity could not grow (index unchanged), PI_ERR_CUDA on a launch
 * failure, PI_ERR_TIMEOUT if an earlier batch reported a device-side timeout.
 */
int pi_execute_batch(pi_index_t* idx, const uint8_t* ops, const uint64_t* keys,
                     const uint64_t* values, uint64_t n, pi_result_t* results,
                     pi_stream_t stream);

/*
 * pi_execute_batch_host -- the same, with HOST arrays. The library copies the inputs
 * to device staging it owns, runs the batch and copies the results back, each step on a
 * stream of its own, with two staging slots: the copies of one call overlap the kernels
 * of the calls before and after it. results_host is complete when `stream` completes
 * (the caller's stream waits for the copy out). The batch is ordered after the index's
 * previous operation; the copy in does not wait for other earlier work on `stream`, so
 * the host arrays must hold the batch when the call is made and stay unchanged (and
 * allocated) until `stream` completes. Pinned host memory makes the copies
 * asynchronous; pageable memory works but serialises them.
 */
int pi_execute_batch_host(pi_index_t* idx, const uint8_t* ops_host, const uint64_t* keys_host,
                          const uint64_t* values_host, uint64_t n, pi_result_t* results_host,
                          pi_stream_t stream);

/*
 * pi_execute_batch_noalloc -- the same as pi_execute_batch, for callers that cannot
 * allocate device memory during a batch. (The paper has no counterpart: this is an
 * interface choice.) Such callers include code that must not block on the CUDA
 * allocator (cudaMalloc/cudaFree can synchronise the device, which a latency-bound
 * serving loop cannot afford) and code running where a memory budget is fixed up front.
 * The per-batch scratch of up to PI_NOALLOC_MAX_BATCH queries comes from one
 * file-scope device array of a fixed size (about 10.9 MB), held by
 * every GPU that loads the library until the process exits; this call allocates nothing.
 *   - n > PI_NOALLOC_MAX_BATCH returns PI_ERR_INVALID_ARG.
 *   - A batch that could need the storage layer to grow returns PI_ERR_OOM with the
 *     index unchanged (create the index with enough storage_capacity, or use
 *     pi_execute_batch for that batch). An index layer that outgrows its capacity is not
 *     grown: its lowest levels are dropped and the results stay exact.
 *   - The first call on a device looks up the array's device address and creates one
 *     event (with that device current); make that first call before any stream capture.
 *   - Every call shares the one array. Calls issued in order on one stream are safe, on
 *     one index or alternating between indices: a call on another index than the
 *     previous call's first makes its stream wait for that call's background rebuild,
 *     which still reads the array. Calls whose work overlaps on the GPU (issued on
 *     different streams without ordering between them) race and must be serialised by
 *     the caller. Nothing in the array needs to start at zero; each batch writes what it
 *     later reads.
 * Results and the resulting key/value set are identical to pi_execute_batch's. The
 * index layer's shape can differ after pi_execute_batch would have grown its capacity
 * (its lowest levels are then dropped here); searches stay exact either way.
 */
#define PI_NOALLOC_MAX_BATCH (1u << 16)
int pi_execute_batch_noalloc(pi_index_t* idx, const uint8_t* ops, const uint64_t* keys,
                             const uint64_t* values, uint64_t n, pi_result_t* results,
                             pi_stream_t stream);

/*
 * pi_flush -- makes `stream` wait (on the device, without blocking the host) until all
 * work the index has in flight has finished. A batch's index-layer rebuild runs in the
 * background on a library-owned stream, as the paper's rebuild daemon does (Section
 * 4.4.4): the next batch, and every other call on the index, waits for it by itself,
 * so this is needed only to include that work in a caller's own timing or ordering.
 */
int pi_flush(pi_index_t* idx, pi_stream_t stream);

/* Releases every device allocation of the index after its pending work. NULL-safe. */
void pi_destroy(pi_index_t* idx);

/* Error code of the last failing pi_create / pi_create_ex on this host thread. */
int pi_last_error(void);

/* Synchronises `stream` and returns PI_OK, or the sticky device-side error
 * (PI_ERR_TIMEOUT / PI_ERR_CUDA) recorded by any batch so far. */
int pi_status(pi_index_t* idx, pi_stream_t stream);

/* Snapshot of the index's shape (synchronises `stream`). */
typedef struct {
    uint64_t size;           /* storage-layer nodes, delete-flagged ones included */
    uint64_t live;           /* live keys */
    uint64_t tombstones;     /* delete-flagged nodes still in the storage layer */
    uint32_t top_level;      /* H: highest level holding a key (1 if only storage) */
    uint32_t bottom_built;   /* lowest materialised index level (pi_config_t.lowest_level,
                                raised when the index layer overflows its capacity) */
    uint32_t smem_low_level; /* lowest level staged in shared memory by the descent */
    uint32_t promote_shift;  /* b, with P = 2^-b */
    uint64_t level_size[34]; /* level_size[l] = live keys with height >= l, l = 1..33 */
    uint64_t storage_capacity;
    uint64_t index_capacity;
    uint64_t batches;        /* batches executed */
    uint64_t rebuilds;       /* index-layer rebuilds run (counts only when known) */
    uint64_t kernel_launches; /* CUDA kernels the batch entry points have launched so far */
    uint64_t incremental_rebuilds; /* rebuilds that updated the previous levels (no storage
                                      re-layout) rather than scanning the storage layer */
    uint64_t owner_checked_writes; /* PI_TEST_OWNER_CHECK: storage-node writes checked */
    uint64_t routed_batches; /* batches that took the small-batch route (one cluster
                                launch each; pi_config_t.small_batches) */
} pi_info_t;
int pi_info(pi_index_t* idx, pi_info_t* out_host, pi_stream_t stream);

/* Live keys, i.e. the size of level 1 (Definition 1), after the batches enqueued on
 * `stream` (synchronises it). Returns PI_OK or, like pi_status, the sticky error. */
int pi_size(pi_index_t* idx, uint64_t* size_out_host, pi_stream_t stream);

/*
 * Failure-path support (no counterpart in the paper).
 * pi_test_fail_allocations: the next `count` device allocations the library makes on the
 *   calling host thread fail as if the device were out of memory (0 clears). The call
 *   that hits one returns PI_ERR_OOM and leaves the index as it was.
 * pi_selftest_wait: launches one CTA that waits, through the bounded look-back the batch
 *   kernels use, for a predecessor that never publishes. The wait gives up after its
 *   spin bound (on a GB300 about 1.4 s), records the timeout in a scratch error word, which
 *   is written to *err_word_host, and the kernel returns. Returns PI_ERR_TIMEOUT when the
 *   bound worked. Allocates and frees 516 B of device memory; synchronises `stream`.
 */
void pi_test_fail_allocations(uint32_t count);
int pi_selftest_wait(uint32_t* err_word_host, pi_stream_t stream);

/* H, the number of levels (Definition 1: level 1 is the storage layer, so H = 1 when no
 * live key reaches level 2), after the batches enqueued on `stream` (synchronises it).
 * Returns H >= 1, or a negative PI_ERR_* code. */
int pi_num_levels(pi_index_t* idx, pi_stream_t stream);

/* Live keys (level 1). *n_out_host = live count; up to cap pairs are written, in key
 * order, to the device arrays keys_out / vals_out. Synchronises `stream`. */
int pi_export(pi_index_t* idx, uint64_t* keys_out, uint64_t* vals_out, uint64_t cap,
              uint64_t* n_out_host, pi_stream_t stream);

/* Level `level` (>= 2) of the index layer as last rebuilt: its keys and, if down_out
 * is not NULL, each key's position in the level below (for the lowest materialised
 * level: its storage-layer position). Device arrays; *n_out_host = the level's size.
 * PI_ERR_NOT_BUILT if the level is not materialised. Synchronises `stream`. */
int pi_export_level(pi_index_t* idx, int level, uint64_t* keys_out, uint32_t* down_out,
                    uint64_t cap, uint64_t* n_out_host, pi_stream_t stream);

/* Test support: the storage layer as it is stored (Definition 1's level 1 with the
 * delete-flagged nodes of Algorithm 4 still in place), positions 0 .. size-1, so a test
 * can check the lowest built level's down pointers (its storage positions) while
 * delete-flagged nodes exist. Up to cap keys and meta bytes (bits 0-5: tower height;
 * bit 7: delete flag) are written to the device arrays keys_out / meta_out (meta_out may
 * be NULL); *n_out_host = size. Synchronises `stream`. Returns PI_OK or the sticky
 * error, like pi_status. */
int pi_export_storage(pi_index_t* idx, uint64_t* keys_out, uint8_t* meta_out, uint64_t cap,
                      uint64_t* n_out_host, pi_stream_t stream);

/*
 * Stage timing, for measurement (no counterpart in the paper). While enabled, each
 * pi_execute_batch records CUDA events between the pipeline's stages, on the stream
 * each stage runs on:
 *   0 pack + radix sort (K0, K1)        4 level layout (K6b)
 *   1 descent + storage locate (K2, K3) 5 index-layer rebuild (K6c; background stream)
 *   2 ownership + apply (K4, K5)        6 the rebuild's writer kernels alone (part of 5)
 *   3 storage merge (K6a)               7 the storage-locate kernel alone (part of 1)
 * The descent's stage excludes its wait for the previous batch's rebuild.
 * pi_profile(idx, 1) starts (and clears) the accumulation; pi_profile(idx, 0) stops it.
 * pi_profile_read synchronises `stream` and writes the summed milliseconds per stage to
 * stage_ms_host[PI_NUM_STAGES] and the number of batches they cover to *batches_host.
 * pi_profile(idx, 2) also times every kernel launch of the batch entry points between
 * two events on its own stream (which serialises the launches it brackets: use it to
 * compare kernels, not to measure throughput). pi_profile_kernels synchronises `stream`
 * and writes one text line per kernel, "<function name>\t<launches>\t<summed ms>\n",
 * NUL-terminated, to buf[cap] (truncated to fit); it returns the length the whole table
 * needs including the NUL, or PI_ERR_INVALID_ARG when level 2 is not on.
 */
#define PI_NUM_STAGES 8
int pi_profile(pi_index_t* idx, int enable);
int pi_profile_read(pi_index_t* idx, double* stage_ms_host, uint64_t* batches_host, pi_stream_t stream);
int pi_profile_kernels(pi_index_t* idx, char* buf, uint64_t cap, pi_stream_t stream);

/*
 * pi_range_search -- range queries (Section 3.2.5) on the index as it stands after the
 * batches enqueued before it on `stream` (read-only: it changes nothing).
 *   lo, hi: device arrays of n inclusive bounds; lo > hi is an empty range; any 64-bit
 *     value is a valid bound (2^64-1 as hi means "to the end").
 *   offsets: device array of n + 1: query i's pairs are [offsets[i], offsets[i + 1]) of
 *     the output, in key order; offsets[n] is the total.
 *   keys_out, vals_out: device arrays of cap pairs (may be NULL when cap is 0). The pairs
 *     of a query are written only when they all fit below cap; the caller reads
 *     offsets[n] and calls again with room for the total if it exceeds cap.
 * n <= PI_MAX_BATCH / 2. Errors as for pi_execute_batch. Enqueued on `stream` like a
 * batch: the arrays are in use until the stream reaches the end of the call.
 */
int pi_range_search(pi_index_t* idx, const uint64_t* lo, const uint64_t* hi, uint64_t n, uint64_t* offsets,
                    uint64_t* keys_out, uint64_t* vals_out, uint64_t cap, pi_stream_t stream);

/*
 * ---------------------------------------------------------------------------------
 * Batching form: one batch for each of many independent indices in one persistent
 * launch. Algorithm 1 runs for every index of the set at once: each CTA (or, for a size
 * class configured so, each thread-block cluster) takes a batch from a device-side queue
 * (largest first) and runs its whole pipeline. The result of
 * every batch is exactly what pi_execute_batch gives for it (Section 4.2: arrival-order
 * semantics per index); the indices stay usable by every single-index entry point.
 * The paper runs one index per NUMA node (Section 4.4.1); many small indices in one
 * launch are this library's extension.
 */
typedef struct pi_multi pi_multi_t;

/* Kernel configuration of one size class: indices whose storage layer has at most
 * 2^max_log2_size nodes take CTAs of `warps` warps (8, 16 or 32) and radix digits of
 * `radix_bits` bits (4 or 8). `cluster` is the number of CTAs that share one batch:
 * 0 or 1 gives each batch one CTA; 2, 4, 8 or 16 give it a thread-block cluster of
 * that many CTAs (on as many SMs), which splits every stage of the batch into one span
 * per CTA and needs warps = 16 or 32 and radix_bits = 8. */
typedef struct {
    uint32_t max_log2_size;
    uint32_t warps;
    uint32_t radix_bits;
    uint32_t cluster;
} pi_multi_class_t;

#define PI_MULTI_MAX_CLASSES 4
#define PI_MULTI_MAX_BATCH (1u << 20) /* queries per batch in the batching form */

typedef struct {
    uint32_t struct_size;   /* sizeof(pi_multi_config_t) */
    uint32_t num_classes;   /* 1..PI_MULTI_MAX_CLASSES, ascending max_log2_size; the
                               last class takes every larger index */
    pi_multi_class_t cls[PI_MULTI_MAX_CLASSES];
} pi_multi_config_t;

/*
 * pi_multi_create -- group `count` indices (made by pi_create / pi_create_ex on the
 * current device) for batched execution. The set refers to the indices, it does not own
 * them: destroy the set before its indices. cfg may be NULL (built-in classes). Returns
 * NULL on error (pi_last_error: PI_ERR_INVALID_ARG for a NULL or repeated index or a bad
 * class, PI_ERR_OOM, PI_ERR_CUDA).
 */
pi_multi_t* pi_multi_create(pi_index_t* const* indices, uint32_t count, const pi_multi_config_t* cfg);

/* One batch for one index of the set. Arrays as for pi_execute_batch (device memory,
 * n <= PI_MULTI_MAX_BATCH, results[n] in arrival order). */
typedef struct {
    uint32_t index;          /* position in the set */
    uint32_t reserved;
    const uint8_t* ops;
    const uint64_t* keys;
    const uint64_t* values;
    uint64_t n;
    pi_result_t* results;
} pi_multi_batch_t;

/*
 * pi_multi_execute -- enqueue `nb` batches (host array of descriptors, at most one per
 * index) on `stream` as one CUDA-graph launch. Returns PI_ERR_INVALID_ARG for a bad
 * descriptor (nothing is enqueued), PI_ERR_OOM / PI_ERR_CUDA when growing an index's
 * capacity fails, or a sticky device error of one of the indices. Results are complete
 * when `stream` reaches the end of the call. The descriptor array may be reused as soon
 * as the call returns.
 */
int pi_multi_execute(pi_multi_t* set, const pi_multi_batch_t* batches_host, uint32_t nb, pi_stream_t stream);

/* Kernels one pi_multi_execute call launches (one persistent kernel per size class in
 * use when its graph was built); 0 before the first call or for NULL. */
uint64_t pi_multi_kernels_per_call(const pi_multi_t* set);

/* Releases the set's own device and host memory (not the indices). NULL-safe. */
void pi_multi_destroy(pi_multi_t* set);

/*
 * ---------------------------------------------------------------------------------
 * Serving form: continuous batching of variable-size requests against one resident
 * index. Clients submit requests (host arrays, copied into a pinned ring at submit: the
 * ring's size is the admission budget, and submit waits while it is full). A dispatcher
 * thread coalesces the queued requests, in arrival order, into batches of at most
 * max_batch queries and keeps up to `slots` batches in flight: batch k+1's inputs are
 * copied to the device while batch k's kernels run, and batch k's results are copied
 * back while batch k+1's kernels run. A batch is Algorithm 1 on the concatenated
 * requests, so every query's result equals the result of running the requests one by
 * one in arrival order (Section 4.2); coalescing changes no result. This answers the
 * latency concern the paper raises for batching (Section 3.2, right after
 * Algorithm 1, and Section 6's batch-size experiments) with a bounded batch and
 * overlapping stages; the serving loop itself is this library's extension.
 * While a server exists, its index must not be used by any other call.
 */
typedef struct pi_server pi_server_t;

typedef struct {
    uint32_t struct_size;    /* sizeof(pi_server_config_t) */
    uint32_t max_batch;      /* queries per coalesced batch, 1..PI_MAX_BATCH (default 2^20) */
    uint32_t slots;          /* batches in flight, 2..8 (default 3) */
    uint32_t reserved;
    uint64_t ring_queries;   /* pinned staging capacity in queries, >= max_batch
                                (default 8 x max_batch) */
} pi_server_config_t;

/* Starts a server on `idx` (current device). cfg may be NULL. NULL on error
 * (pi_last_error: PI_ERR_INVALID_ARG, PI_ERR_OOM, PI_ERR_CUDA). */
pi_server_t* pi_server_create(pi_index_t* idx, const pi_server_config_t* cfg);

/* Queues one request of n (1..max_batch) queries: host arrays as for pi_execute_batch,
 * copied before the call returns. Waits while the ring has no room. *ticket_out gets
 * the request's ticket (consecutive from 1). Returns the server's sticky error, if any. */
int pi_server_submit(pi_server_t* srv, const uint8_t* ops, const uint64_t* keys, const uint64_t* values,
                     uint32_t n, uint64_t* ticket_out);

/* Waits for the oldest uncollected request, which must be `ticket` (tickets are
 * collected in submission order), copies its n results to results_out (host, may be
 * NULL) and its latency in seconds (submission to results in host memory) to
 * *latency_s (may be NULL), and frees its ring space. */
int pi_server_wait(pi_server_t* srv, uint64_t ticket, pi_result_t* results_out, double* latency_s);

typedef struct {
    uint64_t requests;        /* completed since the last reset */
    uint64_t queries;
    uint64_t batches;
    uint32_t max_in_flight;   /* most batches on the GPU at once */
    uint32_t reserved;
    double p50_s, p99_s, max_s;  /* request latency */
    double mean_batch;        /* queries per batch */
} pi_server_stats_t;

/* Statistics of the requests completed since the last reset (reset != 0 starts anew). */
int pi_server_stats(pi_server_t* srv, pi_server_stats_t* out, int reset);

/*
 * pi_server_replay -- load generator: submits nreq requests, request i being the next
 * sizes[i] queries of the host arrays, each at arrival_s[i] seconds after the call
 * starts (non-decreasing), collects them in order on a second thread, and returns when
 * all are done. A request's latency runs from its scheduled arrival (so a late submit
 * counts against the server) to its results in host memory; latency_s_out[nreq] and
 * results_out[sum of sizes] may be NULL.
 */
int pi_server_replay(pi_server_t* srv, const uint8_t* ops, const uint64_t* keys, const uint64_t* values,
                     const uint32_t* sizes, const double* arrival_s, uint32_t nreq, pi_result_t* results_out,
                     double* latency_s_out);

/* Finishes the queued requests, stops the dispatcher and frees the server (not the
 * index). NULL-safe. */
void pi_server_destroy(pi_server_t* srv);

#ifdef __cplusplus
}
#endif

#endif /* PI_H_ */

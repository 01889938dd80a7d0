/*
 * bsort.h -- C ABI of the GB300 block-decomposed sort.
 *
 * The library sorts integer and floating-point key arrays that live in GPU
 * memory, following the scatter / sort / merge paradigm of El-Nashar,
 * "Parallel performance of MPI sorting algorithms on dual-core processor
 * Windows-based systems" (IJDPS 2(3), 2011), Section 3.2 and Figure 1:
 *   scatter (Fig. 1)             the n keys are split into p blocks with
 *                                bounds b_i = floor(i*n/p);
 *   sort    (Fig. 1)             every block is sorted on its own -- here by
 *                                CTA-local tile sorts and in-block merge
 *                                passes in GPU memory;
 *   merge   (Fig. 1;             sorted blocks are merged pairwise, round
 *            Sec. 3.2.2)         after round, into one nondecreasing output.
 * The output does not depend on p; p only changes the schedule.
 *
 * Ordering.  Keys are ordered by an order-preserving unsigned code: signed
 * integers by value, unsigned integers by value, floating point by the IEEE
 * 754-2008 totalOrder predicate (Sec. 5.10): -NaN < -inf < ... < -0 < +0 <
 * ... < +inf < +NaN, NaNs by payload.  Every comparison is an integer one, so
 * results are bit-exact and deterministic.  Pair sorts are stable: equal keys
 * keep their input order, and so do their values.
 *
 * Memory.  Every d_* pointer is a device pointer owned by the caller; the
 * library never frees it.  Input and output may be the same buffer (in-place
 * sort).  Scratch memory (a ping-pong copy of keys and values plus small
 * index arrays, see bs_workspace_bytes) is owned by the handle and grown on
 * demand with cudaMalloc; it is freed by bs_destroy.
 *
 * Streams and errors.  Calls are asynchronous on `stream` (a cudaStream_t
 * passed as void*, NULL = the legacy default stream).  Argument errors are
 * returned synchronously before anything is launched.  Errors the GPU finds
 * (e.g. invalid segment offsets) are recorded in the handle and returned by
 * bs_sync_status.  A handle is not thread safe: use one handle per host
 * thread, and do not run two calls of one handle on different streams at the
 * same time (they share the scratch memory).
 */
#ifndef BSORT_H
#define BSORT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BS_OK = 0,
    BS_ERR_INVALID_ARG = 1,       /* bad pointer, size, p, offsets */
    BS_ERR_UNSUPPORTED_DTYPE = 2, /* key or value dtype not supported */
    BS_ERR_OUT_OF_MEMORY = 3,     /* scratch allocation failed */
    BS_ERR_CUDA = 4,              /* a CUDA runtime call or launch failed */
    BS_ERR_TIMEOUT = 5,           /* a bounded device-side wait gave up */
    BS_ERR_TOO_LARGE = 6          /* request exceeds a fixed capacity (bs_sort_keys_noalloc) */
} bs_status;

typedef enum {
    BS_NONE = -1, /* no values (keys-only) */
    BS_INT32 = 0,
    BS_UINT32 = 1,
    BS_FLOAT32 = 2,
    BS_INT64 = 3,
    BS_UINT64 = 4,
    BS_FLOAT64 = 5
} bs_dtype;

/* Kernel classes reported by the launch statistics. */
typedef enum {
    BS_KERNEL_TILE_SORT = 0, /* sort phase: CTA-local tile sort (1 pass) */
    BS_KERNEL_MERGE = 1,     /* merge pass of sorted runs (1 pass each) */
    BS_KERNEL_PARTITION = 2, /* merge-path split search per merge pass */
    BS_KERNEL_SETUP = 3,     /* scatter bounds, tile map, offset checks */
    BS_KERNEL_CLASSES = 4
} bs_kernel_class;

typedef struct bs_handle bs_handle;

/*
 * Create a handle on CUDA device `device` (the analogue of initialising MPI
 * in Fig. 1).  *h receives the handle.  Errors: INVALID_ARG (h NULL or no such
 * device), CUDA, OUT_OF_MEMORY.
 */
bs_status bs_create(bs_handle **h, int device);

/* Free the handle and its scratch memory (finalising MPI in Fig. 1).  Waits for the
 * handle's outstanding work.  NULL is accepted. */
bs_status bs_destroy(bs_handle *h);

/*
 * Sort n keys of dtype kt from d_in into d_out (nondecreasing), decomposed
 * into p blocks as in Fig. 1: each block sorted on its own, then the blocks
 * merged pairwise (the merge phase).  p = 0 picks p = 1; p > n is clamped to
 * n.  n = 0 is a no-op.  Key dtypes: all of bs_dtype except BS_NONE.
 * Errors (synchronous): INVALID_ARG for n < 0, p < 0, a NULL pointer with
 * n > 0; UNSUPPORTED_DTYPE; OUT_OF_MEMORY; CUDA.
 */
bs_status bs_sort_keys(bs_handle *h, const void *d_in, void *d_out, int64_t n,
                       bs_dtype kt, int64_t p, void *stream);

/*
 * Stable sort of (key, value) pairs: keys d_kin -> d_kout as bs_sort_keys,
 * and each value moves with its key (d_vin -> d_vout).  Values are any 4- or
 * 8-byte type (vt gives the width; the bits are carried unchanged).  Equal
 * keys keep their input order.  Errors as bs_sort_keys; vt == BS_NONE is
 * UNSUPPORTED_DTYPE (use bs_sort_keys).
 */
bs_status bs_sort_pairs(bs_handle *h, const void *d_kin, void *d_kout, const void *d_vin,
                        void *d_vout, int64_t n, bs_dtype kt, bs_dtype vt, int64_t p,
                        void *stream);

/*
 * Batched sort: S independent segments of one key array are sorted in one
 * call (the sort phase of Fig. 1 applied to every segment, no merge across
 * segments).  Segment s is [d_offsets[s], d_offsets[s+1]); d_offsets is a
 * device array of S+1 int64 with d_offsets[0] = 0, d_offsets[S] = n and
 * nondecreasing entries (empty segments allowed).  d_vin / d_vout may be NULL
 * (keys-only, vt = BS_NONE) or carry values (each segment sorted stably).
 * max_seg_len: 0 = unknown, else an upper bound on every segment's length,
 * which lets the library launch fewer merge passes.  Offsets that break these
 * rules, or a segment longer than max_seg_len, are detected on the GPU and
 * reported as INVALID_ARG by bs_sync_status; the output is then undefined but
 * no memory outside the arrays is touched.
 */
bs_status bs_sort_segmented(bs_handle *h, const void *d_kin, void *d_kout, const void *d_vin,
                            void *d_vout, int64_t n, const int64_t *d_offsets, int64_t S,
                            int64_t max_seg_len, bs_dtype kt, bs_dtype vt, void *stream);

/*
 * Gathered batch (the serving layer): like bs_sort_segmented, but segment s
 * reads its len_s = d_offsets[s+1] - d_offsets[s] keys (and values) from
 * d_kin[d_src_offsets[s] ...] of an input array of n_in items, so requests
 * resident anywhere in one buffer are sorted in one call without a gather
 * copy; output segment s is d_kout[d_offsets[s] ...].  d_src_offsets: S
 * int64 on the device.  A source range outside [0, n_in) is reported by
 * bs_sync_status as INVALID_ARG (nothing outside the arrays is read).  The
 * output must not overlap the input ranges it is read from.
 */
bs_status bs_sort_segmented_gather(bs_handle *h, const void *d_kin, int64_t n_in,
                                   const int64_t *d_src_offsets, void *d_kout, const void *d_vin,
                                   void *d_vout, int64_t n, const int64_t *d_offsets, int64_t S,
                                   int64_t max_seg_len, bs_dtype kt, bs_dtype vt, void *stream);

/*
 * Merge phase only (the gather-to-master form of Sec. 3.2.2): d_kin holds
 * `runs` runs that are each already sorted (nondecreasing in the dtype's
 * order); run r is [h_run_offsets[r], h_run_offsets[r+1]).  The runs are
 * merged pairwise, round after round, into d_kout (stable: equal keys keep
 * run order, then position).  h_run_offsets is a HOST array of runs+1 int64
 * with h_run_offsets[0] = 0, h_run_offsets[runs] = n, nondecreasing (checked
 * synchronously: INVALID_ARG); it is read during the call only.  Values
 * optional as in bs_sort_segmented.  Runs that are not sorted give an
 * undefined (but in-bounds) result.  Used by the multi-GPU exchange sort to
 * merge the runs one GPU receives.
 */
bs_status bs_merge_runs(bs_handle *h, const void *d_kin, void *d_kout, const void *d_vin,
                        void *d_vout, int64_t n, const int64_t *h_run_offsets, int64_t runs,
                        bs_dtype kt, bs_dtype vt, void *stream);

/*
 * Host-memory convenience: sort n keys from host buffer h_in into host
 * buffer h_out (may be equal) on the handle's internal stream; returns after
 * the result is in h_out.  When both buffers are page-locked (or registered)
 * and mapped into the GPU's address space -- the coherent host link of a
 * Grace-Blackwell node -- the sort phase reads h_in and the last merge pass
 * writes h_out directly, and every other pass stays in device memory;
 * otherwise (or with BS_OPT_HOST_DIRECT = 0) the keys are copied in, sorted
 * and copied out.  Errors as bs_sort_keys.
 */
bs_status bs_sort_keys_host(bs_handle *h, const void *h_in, void *h_out, int64_t n,
                            bs_dtype kt, int64_t p);

/*
 * Asynchronous host-memory sort: enqueues the copy of h_in into the input
 * buffer of one of the handle's device slots (three by default,
 * BS_OPT_HOST_SLOTS; on an internal copy stream), the sort (as bs_sort_keys:
 * p blocks, Fig. 1; on `stream`) into the slot's output buffer and the copy
 * of the result into h_out (may equal h_in; on a second internal copy
 * stream), and returns.  Successive calls on one handle form a pipeline:
 * call k+1's copy in and call k-1's copy out run on the copy engines while
 * call k sorts, neither waiting for the other, and the sorts of a handle run
 * one after another whatever streams they are given.  h_in must stay
 * unchanged and h_out unread until bs_sync_status(h), which waits for all of
 * the handle's work, returns.  The copies are asynchronous only for
 * page-locked buffers.  Device memory: an input and an output buffer of n
 * keys per slot, besides the workspace.  Errors as bs_sort_keys.
 */
bs_status bs_sort_keys_host_async(bs_handle *h, const void *h_in, void *h_out, int64_t n,
                                  bs_dtype kt, int64_t p, void *stream);

/*
 * Scratch bytes one sort of n keys (value type vt, BS_NONE for none) in S
 * segments/blocks needs; the handle allocates this much on first use.
 */
bs_status bs_workspace_bytes(int64_t n, int64_t S, bs_dtype kt, bs_dtype vt, size_t *bytes);

/*
 * Order keys: d_out[i] (int64, device) receives, for key d_in[i] of dtype kt,
 * a signed 64-bit integer whose order is this library's sort order (the
 * key's order-preserving code: 4-byte codes zero-extended, 8-byte codes with
 * the top bit flipped; floating point by IEEE 754 totalOrder).  Used to cut
 * sorted runs at splitters in the library's order, as the multi-GPU exchange
 * sort's bucketing does (the merge phase of Fig. 1 across processes).  Runs
 * on the current device, asynchronously on `stream`; needs no handle and
 * allocates nothing.  Errors: INVALID_ARG (n < 0, NULL pointer with n > 0),
 * UNSUPPORTED_DTYPE, CUDA.
 */
bs_status bs_order_keys(const void *d_in, int64_t *d_out, int64_t n, bs_dtype kt, void *stream);

/*
 * Device checkers of a sort's result (test infrastructure; no counterpart
 * in the paper, whose correctness criterion -- a nondecreasing permutation
 * of the input, Sec. 3 -- they test in one pass over device memory).
 * code(k) is the key's order-preserving code as a uint64 (4-byte codes
 * zero-extended), the code the sort compares.
 *   first_unsorted: the smallest i, 0 < i < n, with code(k[i-1]) > code(k[i])
 *     where i does not start a segment (d_offsets: S+1 device offsets,
 *     0 = off[0] <= .. <= off[S] = n; NULL: one run), else -1.
 *   first_unstable: with d_idx (device, n payload indices of dtype it:
 *     INT32, UINT32, INT64 or UINT64), the smallest such i with equal codes
 *     and idx[i-1] >= idx[i], else -1 (always -1 without d_idx).
 *   hash_a, hash_b: sum over all keys of mix_a(code) and mix_b(code) mod
 *     2^64, multiset hashes equal for any permutation of the same keys.
 *     mix_a(x): x ^= x >> 33; x *= 0xff51afd7ed558ccd; x ^= x >> 33;
 *       x *= 0xc4ceb9fe1a85ec53; x ^= x >> 33 (MurmurHash3 fmix64).
 *     mix_b(x): x += 0x632be59bd9b4e019; x ^= x >> 29; x *= 0xbf58476d1ce4e5b9;
 *       x ^= x >> 32; x *= 0x94d049bb133111eb; x ^= x >> 29.
 */
typedef struct {
    int64_t first_unsorted;
    int64_t first_unstable;
    uint64_t hash_a, hash_b;
} bs_check_result;

/*
 * Runs the checkers on `stream` (the current device) and waits for them;
 * *result (host memory) receives the outcome.  n = 0 gives -1, -1, 0, 0.
 * It allocates a 32-byte accumulator from the stream-ordered allocator.
 * Errors: INVALID_ARG (result NULL, n < 0, d_keys NULL with n > 0,
 * d_offsets with S < 1), UNSUPPORTED_DTYPE (kt; it when d_idx is given),
 * OUT_OF_MEMORY, CUDA.
 */
bs_status bs_check_keys(const void *d_keys, int64_t n, bs_dtype kt, const int64_t *d_offsets, int64_t S,
                        const void *d_idx, bs_dtype it, bs_check_result *result, void *stream);

/*
 * Grow the handle's scratch now to what one sort of n keys (value type vt,
 * BS_NONE for none) in S blocks or segments needs (bs_workspace_bytes), so
 * that later calls of up to that size and block/segment count allocate
 * nothing: a serving loop reserves its handles' scratch once, before it
 * admits work against the memory left.  Waits for the handle's work first
 * when the scratch has to grow.  *bytes (may be NULL) receives the handle's
 * scratch size afterwards.  Errors: INVALID_ARG (h NULL, n < 0, S < 0),
 * UNSUPPORTED_DTYPE, OUT_OF_MEMORY.
 */
bs_status bs_reserve_workspace(bs_handle *h, int64_t n, int64_t S, bs_dtype kt, bs_dtype vt,
                               size_t *bytes);

/*
 * Wait for the handle's last stream and for every copy out queued by
 * bs_sort_keys_host_async, then return the first error the GPU recorded
 * since the previous call (and clear it), else a pending CUDA error, else
 * BS_OK.
 */
bs_status bs_sync_status(bs_handle *h);

/* Static string naming a status. */
const char *bs_status_str(bs_status s);

/*
 * Launch statistics.  counts[k] (k < BS_KERNEL_CLASSES) receives the number
 * of kernels of class k launched through this handle since creation or the
 * last reset; `bytes[k]` the algorithmic bytes those launches had to move
 * (every pass reads and writes each key and value once), counted on the GPU
 * only while BS_OPT_COUNT_BYTES is 1.  Either array may be NULL.  reset != 0
 * zeroes the counters afterwards.
 */
bs_status bs_launch_stats(bs_handle *h, int64_t *counts, double *bytes, int reset);

/*
 * Per-launch GPU timing.  With enable != 0 the handle records a CUDA event
 * pair around every kernel it launches, on the launching stream.
 * bs_kernel_times waits for those events and returns, per kernel class, the
 * summed milliseconds (ms[k]) and the number of timed launches (n[k]); it
 * then forgets the recorded events.
 */
bs_status bs_set_kernel_timing(bs_handle *h, int enable);
bs_status bs_kernel_times(bs_handle *h, double *ms, int64_t *n);

/*
 * Tuning: tile_log2 selects the tile size T = 2^tile_log2 keys of the sort
 * phase and of the merge passes (supported: 11, 12, 13; 0 = default 12).
 * Returns INVALID_ARG for an unsupported value.
 */
bs_status bs_set_tile_log2(bs_handle *h, int tile_log2);

/*
 * CUDA graphs of whole sorts (the batching layer).  A captured graph replays
 * every launch of one call with no host work per launch.  It owns a private
 * handle whose workspace is sized before capture, so it stays valid however
 * the creating handle is used later.  The graph refers to the buffers and the
 * offsets array given at capture: refill them in place and replay.  A segmented
 * graph is valid for any offsets with the same n, S and max_seg_len bound
 * (segment descriptors are read from device memory at every replay).
 * Capturing does not run the sort.
 *
 * bs_graph_capture_segmented: arguments as bs_sort_segmented; *g receives the
 *   graph.  Errors: INVALID_ARG (n <= 0, S <= 0, NULL pointers),
 *   UNSUPPORTED_DTYPE, OUT_OF_MEMORY, CUDA.
 * bs_graph_capture_keys: arguments as bs_sort_keys (n > 0).
 * bs_graph_launch: replay on `stream` (asynchronous).
 * bs_graph_sync_status: as bs_sync_status, for the graph's launches.
 * bs_graph_destroy: waits for the last replay, frees everything; NULL ok.
 */
typedef struct bs_graph bs_graph;
bs_status bs_graph_capture_segmented(bs_handle *h, const void *d_kin, void *d_kout,
                                     const void *d_vin, void *d_vout, int64_t n,
                                     const int64_t *d_offsets, int64_t S, int64_t max_seg_len,
                                     bs_dtype kt, bs_dtype vt, bs_graph **g);
bs_status bs_graph_capture_keys(bs_handle *h, const void *d_in, void *d_out, int64_t n,
                                bs_dtype kt, int64_t p, bs_graph **g);
bs_status bs_graph_launch(bs_graph *g, void *stream);
bs_status bs_graph_sync_status(bs_graph *g);
bs_status bs_graph_destroy(bs_graph *g);

/* Options of bs_set_option. */
typedef enum {
    BS_OPT_TILE_LOG2 = 0,    /* value: 11, 12 or 13 (0 = default 12), as bs_set_tile_log2 */
    BS_OPT_MERGE_KERNEL = 1, /* value: a bs_merge_kernel */
    BS_OPT_MERGE_VT = 2,     /* keys per consumer thread of the TMA merge: 8, 16 or 32;
                                0 (default) = 32 for 32-bit keys alone, 16 otherwise.
                                Fewer keys per thread = more threads per tile; 8 is
                                not offered for 8192-key merge tiles (16 is used) */
    BS_OPT_WAIT_LIMIT_MS = 3,/* limit of every device-side wait, ms (0 = default 2000):
                                a wait that runs out records BS_ERR_TIMEOUT and the
                                kernel returns, leaving the context usable */
    BS_OPT_TEST_WITHHOLD = 4,/* test hook, for failure-detection tests only: while set,
                                each TMA merge pass withholds one stage of its first CTA,
                                so that CTA's bounded waits run out and the call ends
                                with BS_ERR_TIMEOUT (and an incomplete output) */
    BS_OPT_MERGE_SCHEDULE = 5,/* value: a bs_schedule (bs_sort_keys only) */
    BS_OPT_LOCAL_SORT = 6,   /* value: a bs_local_sort (keys-only sorts; pair sorts always
                                use the stable MERGE tile sort) */
    BS_OPT_MERGE_TILE_LOG2 = 7,/* merge-pass tile 2^value keys: 0 (default) = the sort tile,
                                or 11 .. the sort tile's log2; smaller merge tiles use less
                                shared memory, so more CTAs fit per SM */
    BS_OPT_MERGE_CONSUMER = 8,/* TMA merge consumers: 0 (default) each thread finds its own
                                merge-path split and merges its VT outputs sequentially;
                                1 each warp merges a slice with a bitonic merger over
                                registers, shuffles and a shared-memory transpose */
    BS_OPT_HOST_DIRECT = 9,  /* bs_sort_keys_host: 1 (default) reads and writes page-locked
                                host buffers directly from the kernels; 0 always copies
                                through device memory */
    BS_OPT_COUNT_BYTES = 10, /* 1: the kernels add every launch's algorithmic bytes to the
                                handle's counters (one atomic per tile), which
                                bs_launch_stats reports; 0 (default): nothing is counted
                                and `bytes` stays at what earlier counted sorts added */
    BS_OPT_MERGE_PERSISTENT = 11,/* every merge pass of a sort (the in-block levels and
                                the merge phase's rounds) in ONE persistent launch whose
                                CTAs take merge tiles from a work queue in device memory,
                                each tile starting once the runs it reads are complete:
                                1 (default) when a level holds a batch of tiles for every
                                resident CTA (from about 2^25 keys at 8192-key merge
                                tiles; smaller sorts run faster per pass), 2 always, 0
                                never (one partition and one merge launch per pass).  It
                                applies with the default merge consumer and keys per
                                thread, the tree schedule and 16-byte aligned buffers */
    BS_OPT_LENGTH_CLASSES = 12,/* 1 (default): in keys-alone sorts with the MERGE tile sort
                                and the tree schedule, every block or segment of 1 .. 1024
                                keys (512 at 2048-key tiles) is sorted whole by one warp
                                inside the sort-phase launch instead of occupying a tile
                                of its own (with at most 262,144 blocks or segments); 0:
                                every block or segment is cut into tiles */
    BS_OPT_HOST_SLOTS = 13   /* slots of bs_sort_keys_host_async: 3 (default, 0) or 2
                                (two fewer device buffers of n keys; the copy out of
                                call k-2 then gates the sort of call k).  A change
                                first waits for the handle's work, as bs_sync_status,
                                and returns its status */
} bs_option;

/* Sort-phase tile sorts, after the paper's three local sorts:
 * MERGE (default): register bitonic network + merge rounds (merge sort, Fig. 3);
 * BUBBLE: odd-even transposition over the tile (adjacent exchange, Fig. 2), O(T^2);
 * QUICK: CTA quick sort with Fig. 4's middle pivot and '< pivot' partition
 *   (quadratic on heavy duplicates, like the original). */
typedef enum { BS_LOCAL_MERGE = 0, BS_LOCAL_BUBBLE = 1, BS_LOCAL_QUICK = 2 } bs_local_sort;

/* Merge-phase schedules of bs_sort_keys (same output, different passes):
 * TREE (default): ceil(log2 p) rounds merging pairs of sorted runs.
 * ODDEVEN: Fig. 1 read literally -- p compare-split rounds alternating
 *   between block pairs (0,1),(2,3).. and (1,2),(3,4)..; every block gets
 *   the capacity ceil(n/p) (the shorter ones padded with +infinity), which
 *   p rounds need to sort unequal blocks.  p passes instead of log2 p. */
typedef enum { BS_SCHEDULE_TREE = 0, BS_SCHEDULE_ODDEVEN = 1 } bs_schedule;

/* Merge-pass kernels.  AUTO uses the TMA pipeline when the tile's stages fit
 * two CTAs per SM and every buffer is 16-byte aligned; TMA uses it whenever
 * it fits (still falling back on misaligned buffers); SIMPLE never. */
typedef enum { BS_MERGE_AUTO = 0, BS_MERGE_SIMPLE = 1, BS_MERGE_TMA = 2 } bs_merge_kernel;

/* Set one tuning option of the handle; INVALID_ARG for an unknown option or
 * an unsupported value.  Results never depend on options, only speed does. */
bs_status bs_set_option(bs_handle *h, bs_option opt, int64_t value);

/*
 * bs_sort_keys_noalloc -- the paper has no counterpart; this is a service
 * for callers that must not allocate GPU memory while they sort (a latency-
 * critical path where cudaMalloc/cudaFree could stall the device, a plug-in
 * whose host framework owns all device memory, a fixed start-up budget).
 *
 * It sorts like bs_sort_keys (same passes, same bit-exact output) but takes
 * no handle and allocates nothing: its scratch is one fixed array compiled
 * into the library, BS_NOALLOC_MAX_KEY_BYTES plus 64 KiB, which every GPU that
 * loads the library holds until the process exits.  The caller still passes
 * the input and output buffers (device pointers, may be equal).
 *
 * Limits: n * sizeof(key) <= BS_NOALLOC_MAX_KEY_BYTES (2^20 four-byte keys or
 * 2^19 eight-byte keys) and p <= BS_NOALLOC_MAX_BLOCKS after clamping (p = 0
 * means 1, p > n means n).  Larger requests return BS_ERR_TOO_LARGE before
 * any GPU work.  Other errors: INVALID_ARG (n < 0, p < 0, NULL pointer with
 * n > 0), UNSUPPORTED_DTYPE, CUDA (a launch failed).
 *
 * It runs on the calling thread's current CUDA device, asynchronously on
 * `stream`.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) and keeps it for the life of the process;
 * make that first call before any stream capture, and do not use the entry
 * point across a cudaDeviceReset (the array may then live elsewhere).  All
 * calls share the one array, which keeps the last call's contents (nothing
 * in it needs to start at zero): calls whose GPU work overlaps in time
 * (other streams or host threads on the same device) race and corrupt each
 * other's output, so serialise them.
 *
 * Device-side errors are not reported: the call returns before its kernels
 * run and keeps no state to query.  The only one its kernels can meet is a
 * bounded wait running out (BS_ERR_TIMEOUT with a handle; 2 s, a GPU stalled
 * that long), which leaves the output incomplete.  Callers that need it
 * reported use bs_sort_keys and bs_sync_status.
 */
#define BS_NOALLOC_MAX_KEY_BYTES (4u << 20)
#define BS_NOALLOC_MAX_BLOCKS 1024
bs_status bs_sort_keys_noalloc(const void *d_in, void *d_out, int64_t n, bs_dtype kt, int64_t p,
                               void *stream);

#ifdef __cplusplus
}
#endif
#endif /* BSORT_H */

/*
 * bqs.h -- C ABI of the GB300 (sm_103a) data-parallel BlockQuicksort library.
 *
 * The method is BlockQuicksort (Edelkamp & Weiss, arXiv 1604.06697): Quicksort
 * whose partitioning step first compares a whole block of keys with the pivot,
 * keeps the outcomes in a buffer, and only then moves the keys (Sec. 3,
 * Algorithm 3).  Here a block is a tile of keys held by one thread block; the
 * comparison outcomes live in registers, local offsets come from warp ballots
 * and population counts, tile offsets from a block scan, and each tile reserves
 * its output ranges with one atomic before it scatters into a second buffer.
 * Quicksort's main loop (Sec. 2, Algorithm 1) runs level by level over all
 * unfinished segments at once; segments of at most the small-segment cutoff are
 * finished by an in-shared-memory sorting network, standing in for the paper's
 * Insertionsort.
 *
 * Conventions shared by every call
 *   - Keys live in device memory and are owned by the caller.  Pointers to keys,
 *     payloads and outputs must be 16-byte aligned (BQS_ERR_INVALID otherwise).
 *   - dtype: BQS_INT32, BQS_INT64 or BQS_FLOAT64.  float64 keys are ordered by the
 *     total order ord(x) = bits(x) ^ (sign ? ~0 : 1<<63): IEEE "<" on non-NaN
 *     values except that -0.0 sorts before +0.0.  NaN keys are not supported
 *     (the result is then an unspecified permutation of the input).
 *   - n is a key count; 0 <= n < 2^32.  n = 0 and n = 1 are successful no-ops.
 *   - stream is a cudaStream_t passed as an opaque pointer (NULL = the legacy
 *     default stream).  Sorts are asynchronous on it unless stated otherwise.
 *   - Scratch memory (a second key buffer and the segment work lists) comes from
 *     the buffer given to bqs_set_workspace when one is set and large enough,
 *     otherwise from cudaMallocAsync on `stream` (returned with cudaFreeAsync
 *     on the same stream before the call returns).
 *   - Return value: BQS_OK (0) or a negative bqs_status; bqs_status_string()
 *     gives a description, including the CUDA error text for BQS_ERR_CUDA.
 *   - Calls are thread-safe with respect to each other unless they share a
 *     workspace set by bqs_set_workspace.
 */
#ifndef BQS_H_
#define BQS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void* bqs_stream_t; /* a cudaStream_t */

typedef enum { BQS_INT32 = 0, BQS_INT64 = 1, BQS_FLOAT64 = 2 } bqs_dtype;

typedef enum {
  BQS_OK = 0,
  BQS_ERR_INVALID = -1,     /* bad argument (size, alignment, dtype, overlap, offsets) */
  BQS_ERR_NOMEM = -2,       /* scratch memory could not be obtained */
  BQS_ERR_CUDA = -3,        /* a CUDA call or kernel launch failed */
  BQS_ERR_TIMEOUT = -4,     /* a device-side bounded wait ran out */
  BQS_ERR_UNSUPPORTED = -5, /* option or combination not provided */
  BQS_ERR_TOO_LARGE = -7    /* bqs_sort_noalloc: n above its fixed scratch */
} bqs_status;

/* A pivot value for bqs_partition.  dtype selects the member of v that is read. */
typedef struct {
  int32_t dtype;
  int32_t reserved; /* must be 0 */
  union {
    int32_t i32;
    int64_t i64;
    double f64;
  } v;
} bqs_pivot;

/*
 * bqs_partition -- one partitioning step with a caller-given pivot.
 * Paper: Sec. 2 ("Quicksort and improvements": the partitioner leaves elements
 * <= pivot on the left and >= pivot on the right) and Sec. 3 / Algorithm 3 (the
 * block-wise scan-then-rearrange procedure), done by all tiles at once.
 *
 *   keys   device, n keys of pivot->dtype, read only.
 *   n      number of keys.
 *   pivot  host pointer to the pivot value and its dtype.
 *   out    device, n keys, written: out[0, *split) holds exactly the keys < pivot,
 *          out[*split, n) the keys >= pivot (the keys == pivot come first in it).
 *          The order inside each side is unspecified.  out must not overlap keys.
 *   split  host pointer; receives count(keys < pivot).
 * Synchronous: returns after `stream` has completed the work.
 */
int bqs_partition(const void* keys, int64_t n, const bqs_pivot* pivot, void* out,
                  int64_t* split, bqs_stream_t stream);

/*
 * bqs_sort -- sorts keys[0, n) ascending, in place.
 * Paper: Sec. 2 / Algorithm 1 (Quicksort main loop: choose a pivot, partition,
 * recurse on both sides with the pivot excluded), Sec. 3 / Algorithm 3 (block
 * partitioning), Sec. 2 and Sec. 4 (median-of-3 / median-of-sqrt(n) pivots,
 * Introsort depth limit 2 log n + 3, small-array stopper).
 * Asynchronous on `stream`.
 */
int bqs_sort(void* keys, int64_t n, int32_t dtype, bqs_stream_t stream);

/*
 * bqs_sort_segmented -- sorts every segment [seg_offsets[i], seg_offsets[i+1])
 * of keys on its own, in place, i = 0 .. nseg-1, all in one level-synchronous
 * pass over all segments (the batching of small arrays of Sec. 4, "Experiments").
 *   seg_offsets  device, nseg+1 int64 values; must be non-decreasing with
 *                seg_offsets[0] >= 0.  Empty segments are allowed.  A violation
 *                found on the device is reported as BQS_ERR_INVALID.
 * The host reads seg_offsets[nseg] once to size the scratch memory.
 */
int bqs_sort_segmented(void* keys, const int64_t* seg_offsets, int64_t nseg, int32_t dtype,
                       bqs_stream_t stream);

/*
 * bqs_sort_batched -- the segmented sort for batches: like bqs_sort_segmented, but
 * the caller states n = seg_offsets[nseg] (the total key count, used to size the
 * scratch), so the call itself never reads device memory back.  When `stream` is
 * being captured into a CUDA graph, the whole level loop is captured as a device-
 * side loop (a conditional while node; each iteration is one level of persistent
 * kernels over all segments), so one graph launch sorts the whole batch with no
 * host involvement.  Outside capture it behaves like bqs_sort_segmented.  Errors
 * found on the device inside a captured loop (decreasing offsets) stop the loop
 * and are not reported back.  bqs_sort and bqs_sort_pairs capture the same way.
 *   n             number of keys in the array, must equal seg_offsets[nseg].
 *   seg_offsets   device, nseg+1 int64, non-decreasing, seg_offsets[0] >= 0.
 */
int bqs_sort_batched(void* keys, int64_t n, const int64_t* seg_offsets, int64_t nseg,
                     int32_t dtype, bqs_stream_t stream);

/*
 * bqs_sort_pairs -- sorts (keys[i], vals[i]) pairs in place, ordered
 * lexicographically by (key, payload), so the result is unique when payloads
 * are distinct.  Paper: the same method as bqs_sort applied to a wider element
 * (Sec. 4 sorts the 84-byte Record element by its first field the same way).
 *   vals  device, n uint32 payloads, moved with their keys.
 */
int bqs_sort_pairs(void* keys, uint32_t* vals, int64_t n, int32_t dtype, bqs_stream_t stream);

/*
 * bqs_sort_noalloc -- bqs_sort for callers that cannot allocate device memory when
 * they sort (for example a service that reserves all of its GPU memory at start-up
 * and must not grow it or fail with out-of-memory mid-request, or code running
 * inside a framework whose allocator owns the device memory).  The paper has no
 * counterpart; this is a deployment variant of bqs_sort with the same result.
 *
 *   keys, n, dtype, stream  as for bqs_sort; keys is the caller's device array.
 *   Limit: n <= 2^20 keys (any dtype).  Larger n returns BQS_ERR_TOO_LARGE without
 *          touching the GPU; so do option settings whose work lists would not fit.
 * Scratch: a fixed 16 MiB array in the library's device data (allocated when the
 * library is loaded, held by every GPU that loads it until the process exits).  No
 * device or pinned host memory is allocated or freed: no cudaMalloc, cudaMallocAsync,
 * cudaMallocHost or cudaFree call.  The first call on a device looks up that array's
 * device address for
 * the device (cudaGetSymbolAddress) and sets up the kernels; make that first call
 * before any stream capture.  A call on a stream that is being captured into a CUDA
 * graph returns BQS_ERR_UNSUPPORTED and enqueues nothing (the caller's capture stays
 * valid).  All calls share the one array and every call starts
 * by clearing the parts it relies on, so earlier contents do not matter, but calls
 * whose work overlaps on the GPU (different streams or threads at the same time)
 * race on it: serialise them.  Synchronous with respect to `stream` between
 * partition levels, like bqs_sort.
 */
int bqs_sort_noalloc(void* keys, int64_t n, int32_t dtype, bqs_stream_t stream);

/* Keys of wide elements for bqs_sort_records. */
typedef enum {
  BQS_KEY_I32_FIELD = 0,   /* the int32 field at key_offset (the paper's Record type) */
  BQS_KEY_F64_SQNORM = 1   /* squared Euclidean norm of the key_count doubles starting at
                              key_offset (the paper's Vector type, compared by its norm),
                              summed in component order with every product and sum
                              rounded to double (no fused multiply-add) */
} bqs_record_key;

/*
 * Sorts n fixed-size records in place by a key taken from each record: the wide
 * element types of Sec. 4 ("Record": 21 ints compared by the first one; "Vector": 10
 * doubles compared by their norm).  The sort is indirect: each record's key is paired
 * with its index, the (key, index) pairs are sorted like bqs_sort_pairs, and every
 * record is then moved once to its sorted place.  Records with equal keys keep their
 * input order (the index breaks ties), so the output is unique.
 *
 *   records       device, n * record_bytes bytes, caller-owned, sorted in place;
 *                 4-byte aligned (8-byte aligned for BQS_KEY_F64_SQNORM)
 *   record_bytes  a multiple of 4 (of 8 for BQS_KEY_F64_SQNORM)
 *   key_kind      a bqs_record_key; key_offset: byte offset of the key (component)
 *                 in a record, aligned to its type; key_count: doubles in the norm
 *                 (ignored for BQS_KEY_I32_FIELD)
 * Scratch (keys, indices and one copy of the records) comes from cudaMallocAsync on
 * `stream` and is returned on it.  n <= 2^32-1.  Errors: BQS_ERR_INVALID for bad
 * sizes, offsets or alignment; BQS_ERR_NOMEM; BQS_ERR_CUDA.  NaN components are outside
 * the contract.  Synchronous with respect to `stream` between partition levels, like
 * bqs_sort.
 */
int bqs_sort_records(void* records, int64_t n, int32_t record_bytes, int32_t key_kind,
                     int32_t key_offset, int32_t key_count, bqs_stream_t stream);

/* Process-wide options, read at the start of each call. */
typedef enum {
  BQS_OPT_PIVOT = 0,        /* pivot rule (Sec. 4, "Different Pivot Selection Methods"):
                               0 = median-of-3 of first, middle, last (default);
                               1 = median-of-sqrt(n) (median-of-5-medians-of-5 below
                               20000 keys); 2 = median-of-5; 3 = median-of-23;
                               4 = median-of-3-medians-of-3; 5 = median-of-3-medians-
                               of-5; 6 = median-of-5-medians-of-5.  Samples are equally
                               spaced keys; every rule uses median-of-3 below 64 keys */
  BQS_OPT_SMALL_CUTOFF = 1, /* small-segment cutoff C, 2 .. 4096 (default 2048); key-value
                               sorts and BQS_OPT_SMALL_SORT = 1 use at most 2048 */
  BQS_OPT_DEPTH_LIMIT = 2,  /* < 0: 2*floor(log2 n)+3 (default); else this level count */
  BQS_OPT_TIMING = 3,       /* 1: time every partition launch with CUDA events; the call
                               waits for its last one and reports the sum in partition_ms;
                               2 (sorts of the host-driven loop): the same events, but
                               the call never waits for them; bqs_timing_collect() sums
                               them later (partition_ms of the call stays 0) */
  BQS_OPT_TILE = 4,         /* partition tile variant: 0 = default, 1..N autotuner choices */
  BQS_OPT_LOCAL_CUTOFF = 5, /* segments up to this size are partitioned down to the small
                               cutoff inside one thread block's shared memory (one HBM
                               read and write for those levels); -1 = as large as one
                               block holds (8192 keys for 32-bit keys, 4096 otherwise);
                               0 = off, the default; ignored below a small cutoff of 256 */
  BQS_OPT_WAIT_LIMIT = 6,   /* polls before a bounded device-side wait gives up and the
                               call returns BQS_ERR_TIMEOUT (default 2^26, seconds) */
  BQS_OPT_TEST_STALL = 7,   /* failure-path testing: 1 makes the first partition launch
                               of a sort leave one tile unrequested, so its bounded wait
                               runs out (the call returns BQS_ERR_TIMEOUT, the device
                               stays usable; the keys are then unspecified) */
  BQS_OPT_LEVEL_LOOP = 8,   /* 0 (default): after every level the host reads the next
                               level's work counts and sizes its launches to them;
                               1: every kernel reads its counts on the device and the
                               host keeps up to 4 levels enqueued ahead, checking a
                               pinned per-level flag a few levels behind (sorts and
                               segmented sorts; bqs_partition and bqs_sort_noalloc
                               always use 0) */
  BQS_OPT_SMALL_SORT = 9,   /* sorting network for segments of 257 .. small-cutoff keys:
                               0 (default) = key-only: one warp per segment up to 1024
                               (512 for 64-bit keys) keys and one 64-thread (32-bit) or
                               128-thread (64-bit) block above; key-value: the pairs
                               packed into 64-bit keys ((ord(key) - min) << 32 |
                               payload) where the segment's key range allows (always
                               for 32-bit keys), one 256-thread block otherwise;
                               1 = one 256-thread block per segment. */
  BQS_OPT_OVERLAP = 10,     /* 1: the sorting networks of each level run on a second
                               stream of the library's, beside the next partition
                               levels (they touch disjoint key ranges); the call's
                               stream waits for them before the call returns.  0 (the
                               default): everything on the caller's stream.  Used when
                               the host reads the counts after every level. */
  BQS_OPT_LOCAL_SORT = 11,  /* with BQS_OPT_LOCAL_CUTOFF on, key-only sorts and
                               BQS_OPT_SMALL_SORT = 0: the block that partitions a
                               segment in shared memory also sorts up to this many of
                               its finished sub-segments there (the same warp-group
                               networks), so the segment costs one HBM read and one
                               write; further ones, and all with 0, go back to HBM for
                               the network kernels.  0 .. 128, default 0 (measured
                               slower: the block's load, partition and network phases
                               run one after another at 2 blocks per SM) */
  BQS_OPT_COOP_MAX = 12     /* single-array key-only sorts (bqs_sort) of more than the
                               small cutoff and at most this many keys (and fewer than
                               2^24) run every level in one cooperative launch (all
                               blocks resident, one bounded grid-wide barrier per level,
                               the networks after the last level) instead of the
                               host-driven level loop; the call then reads the control
                               block back once, at its end, and its scratch holds the
                               network runs and fills of every level.  0 = never (the
                               default; the autotuner offers it up to 2^22 keys, and at
                               2^20 keys it is faster than the host loop, at 2^22
                               slower).  Not used on a stream that is being captured, by
                               bqs_sort_noalloc, with BQS_OPT_LEVEL_LOOP = 1,
                               BQS_OPT_SMALL_SORT = 1 or local partitioning on, or when
                               the device refuses the cooperative launch (the host loop
                               runs instead). */
} bqs_option;

int bqs_set_option(int32_t opt, int64_t value);
int bqs_get_option(int32_t opt, int64_t* value);

/* Bytes of scratch a call needs: n keys, nseg segments (0 for a single array). */
int bqs_workspace_bytes(int64_t n, int32_t dtype, int32_t with_payload, int64_t nseg,
                        int64_t* bytes);

/*
 * Sets (ptr != NULL) or clears (ptr == NULL) a caller-owned device workspace used
 * by later calls that fit into it.  The caller keeps ownership, must keep it alive
 * while calls that may use it are in flight, and must not let two such calls run
 * concurrently.
 */
int bqs_set_workspace(void* ptr, int64_t bytes);

/* Counters of the calling thread's last sort call. */
typedef struct {
  int64_t levels;            /* partition levels run */
  int64_t partition_launches;
  int64_t active_keys;       /* sum over levels of keys in partitioned segments */
  int64_t moved_keys;        /* of those, keys scattered (< or > pivot) */
  int64_t equal_keys;        /* keys found equal to their segment's pivot */
  int64_t small_segments;    /* segments finished by the small-segment sort */
  int64_t small_keys;
  int64_t local_segments;    /* segments finished inside one thread block */
  int64_t local_keys;
  int64_t fallback_pivots;   /* depth-limit fallbacks */
  int64_t kernel_launches;   /* kernels this library launched for the call */
  double partition_ms;       /* sum of timed partition launches (BQS_OPT_TIMING) */
  double partition_bytes;    /* algorithmic bytes of those launches */
  double coop_ms;            /* the cooperative launch's duration (BQS_OPT_TIMING), else 0 */
} bqs_stats;

int bqs_get_stats(bqs_stats* out);

/*
 * bqs_timing_collect -- with BQS_OPT_TIMING = 2, the summed duration (ms) of the
 * partition launches that had work in the calling thread's sorts on the current device
 * since the last collect, and how many there were.  Waits for those launches to end
 * (call it after synchronising the streams the sorts ran on).  Either pointer may be
 * NULL.
 */
int bqs_timing_collect(double* ms, int64_t* launches);

/* Static description of a status code (thread-local detail for BQS_ERR_CUDA). */
const char* bqs_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* BQS_H_ */

// Shared definitions of the sm_103a BlockQuicksort kernels and their host driver.
//
// Data layout in HBM
//   key[0]  the caller's keys (final output of sorts)
//   key[1]  a second key buffer of the same size (ping-pong partner)
//   val[*]  the same for uint32 payloads of key-value sorts
// A segment is a contiguous index range [off, off+len) whose keys sit in key[parity].
// One partition level moves every key of every large segment from key[parity] into
// key[parity^1]; finished keys (the class equal to a pivot, and small segments after
// their sorting network) are written straight into the final buffer.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bqs {

// ---- key types ---------------------------------------------------------------------
// Keys travel as raw bits U and are compared through an order-preserving unsigned
// image ord(x): one unsigned comparison serves int32, int64 and float64.  For float64,
// ord(x) = bits ^ (sign ? ~0 : 1<<63), a total order equal to IEEE "<" on non-NaN
// values except -0.0 < +0.0.

struct KeyI32 {
  using U = uint32_t;
  static constexpr int kDtype = 0;
  __host__ __device__ static __forceinline__ U ord(U x) { return x ^ 0x80000000u; }
  __host__ __device__ static __forceinline__ U unord(U x) { return x ^ 0x80000000u; }
};

struct KeyI64 {
  using U = uint64_t;
  static constexpr int kDtype = 1;
  __host__ __device__ static __forceinline__ U ord(U x) { return x ^ (1ull << 63); }
  __host__ __device__ static __forceinline__ U unord(U x) { return x ^ (1ull << 63); }
};

struct KeyF64 {
  using U = uint64_t;
  static constexpr int kDtype = 2;
  __host__ __device__ static __forceinline__ U ord(U x) {
    U m = (U)((int64_t)x >> 63);           // all ones for negative values
    return x ^ (m | (1ull << 63));
  }
  __host__ __device__ static __forceinline__ U unord(U x) {
    U m = (U)((int64_t)x >> 63);           // all ones when the order image has its top bit
    return x ^ (~m | (1ull << 63));
  }
};

// Strict order on (ord key, payload); payloads only take part for key-value sorts.
template <bool PAIRS, class U>
__device__ __forceinline__ bool elem_less(U ka, uint32_t va, U kb, uint32_t vb) {
  if constexpr (PAIRS) return ka < kb || (ka == kb && va < vb);
  else return ka < kb;
}

// ---- work lists ------------------------------------------------------------------

// A segment still to be partitioned.
struct Seg {
  int64_t off;
  int64_t len;
  uint64_t pkey;    // pivot: raw key bits (zero-extended)
  uint32_t pval;    // pivot payload (key-value sorts)
  int32_t depth;    // partition levels above this segment
  int32_t parity;   // its keys are in key[parity]
  uint32_t tile0;   // first tile of this segment in the level's tile space
};

// A segment to be finished by one thread block (small-segment sort).
struct Run {
  int64_t off;
  int64_t len;
  int32_t parity;
  int32_t pad;
};

// A range of keys equal to a segment's pivot: written with the pivot value.
struct Fill {
  int64_t off;
  int64_t len;
  uint64_t pkey;
  uint32_t pval;
  uint32_t tile0;
};

// Counts of the lists that one level produces (count | tiles << 32 where tiled).
struct ListCounts {
  unsigned long long large;
  unsigned long long fill;
  unsigned long long large_keys;  // sum of the large segments' lengths
  unsigned int small;
  unsigned int tiny;    // small segments of at most kWarpSortMax keys
  unsigned int todo;    // large segments whose pivot k_pivot chooses
  unsigned int local;
  unsigned int group;   // small segments above the one-warp size (key-only sorts)
  unsigned int big;     // small segments above kMaxSmall keys (key-only sorts)
};

struct Ctrl {
  ListCounts lists[2];
  int status;
  int level;          // current level when the level loop runs on the device
  unsigned long long moved_keys;
  unsigned long long equal_keys;
  unsigned long long small_segs;
  unsigned long long small_keys;
  unsigned long long local_segs;
  unsigned long long local_keys;
  unsigned long long fallbacks;
  // device-driven level loop (host enqueues levels ahead)
  int more[8];                      // per level (mod 8): another level has work
  unsigned long long levels_run;    // levels that partitioned something
  unsigned long long active_total;  // sum of partitioned keys over those levels
  unsigned long long local_runs;    // segments partitioned by one block in shared memory
  unsigned long long small_runs;    // segments finished by the sorting networks
  // grid-wide barrier of the cooperative single-launch sort
  unsigned int bar_count;           // blocks arrived at the current barrier
  unsigned int bar_gen;             // barriers completed
  // k_bookkeep with a host copy: blocks finished (the last one copies the block out)
  unsigned int bk_done;
  unsigned int bk_pad;
  // Single-launch sort: the network runs and pivot-class fills of every level, kept
  // until the end of the launch (`small` counts the runs of all four sizes, `fill`
  // the fills as count | tiles << 32).
  ListCounts acc;
};

struct Bufs {
  void* key[2];
  uint32_t* val[2];
  void* final_key;
  uint32_t* final_val;
};

struct Lists {
  Seg* large[2];
  unsigned long long* cursor[2];  // per large segment: (#< pivot) | (#> pivot) << 32
  unsigned long long* tdone[2];   // per large segment: finished tiles' counts (fused bookkeeping)
  Run* small[2];
  Run* tiny[2];
  Run* group[2];
  Run* big[2];
  uint32_t* todo[2];              // slots of large segments waiting for k_pivot
  Run* local[2];
  Fill* fill[2];
  uint32_t cap_large, cap_run, cap_fill;
};

struct Params {
  Bufs b;
  Lists l;
  Ctrl* ctrl;
  int p;              // parity of the lists consumed by this level
  int pivot_rule;     // BQS_OPT_PIVOT: 0 = median-of-3, 1 = median of a sqrt(n) sample, 2..6 (Sec. 4)
  int small_cutoff;   // segments of at most this many keys go to the sorting network
  int local_cutoff;   // segments of at most this many keys are finished by one block
  int depth_limit;    // partition levels before the depth fallback pivot
  int route_children; // 0: a single partition step (no recursion)
  int tile;           // keys per partition tile (for tile counts)
  int device_loop;    // 1: the level (and its parity) is read from ctrl->level
  int64_t n_keys;     // length of the key arrays
  uint32_t wait_limit;  // polls before a bounded device-side wait gives up
  int test_stall;       // failure-path test: one tile is never requested
  int small_sort;       // 0: warp / warp-group networks for key-only sorts; 1: 256-thread blocks
  int group_min;        // small segments longer than this go to the `group` list
  int local_sort;       // > 0: the single-block local partitioning sorts up to this many
                        // of a segment's leaves itself (at most kLocalSortCap)
  // Network launches on a second stream take their list lengths from here (the
  // device-side counts of their lists may already be cleared for the next level).
  int fixed_counts;
  uint32_t n_tiny, n_small, n_group, n_big;
  unsigned long long n_fill;   // fill list (count | tiles << 32) for k_fill
  // Non-null: the level's last bookkeeping copies the control block here (host-mapped
  // memory), so the host reads a level's counts without a separate copy launch.
  Ctrl* ctrl_host;
  // Non-null (single-launch sort): network runs of every size and pivot-class fills
  // are appended to one list each, counted here, instead of the level's lists.
  ListCounts* net_acc;
};

__device__ __forceinline__ void clear_counts(ListCounts* l) {
  l->large = 0; l->fill = 0; l->large_keys = 0;
  l->small = 0; l->tiny = 0; l->todo = 0; l->local = 0; l->group = 0; l->big = 0;
}

// Parity of the lists the current level consumes: given by the host when it drives
// the level loop, read from the control block when the loop runs on the device.
__device__ __forceinline__ int level_parity(const Params& P, int host_p) {
  return P.device_loop ? (*(volatile int*)&P.ctrl->level & 1) : host_p;
}

// Tiles of a segment start at its first key rounded down to a 16-byte group (4 keys):
// tile k covers [tile_origin(off) + k*tile, + tile) clipped to the segment, so only the
// first tile can start before the segment and only the last one can end early.
__host__ __device__ __forceinline__ int64_t tile_origin(int64_t off) { return off & ~(int64_t)3; }
__host__ __device__ __forceinline__ int64_t tile_count(int64_t off, int64_t len, int tile) {
  return (off + len - tile_origin(off) + tile - 1) / tile;
}

// Device status codes (mirrors the public bqs_status values).
constexpr int kStatusInvalid = -1;
constexpr int kStatusTimeout = -4;   // a bounded device-side wait gave up
constexpr int kStatusOverflow = -6;  // an internal list overflowed its capacity

constexpr int kFillTile = 8192;      // keys per fill task
constexpr int kMaxSmall = 2048;      // largest small-segment cutoff of key-value sorts
constexpr int kMaxSmallKeys = 4096;  // largest small-segment cutoff of key-only sorts
constexpr int kWarpSortMax = 256;    // small segments up to this length are sorted by one warp
constexpr int kMaxSample = 511;      // largest pivot sample
constexpr int kInlineFill = 32;      // pivot-class runs up to this length are written inline

}  // namespace bqs

// Internal declarations shared by the C-ABI front end (bqs_api.cu) and the per-dtype
// driver translation units.
#pragma once

#include <cstdint>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

namespace bqs {

struct Ctrl;

constexpr int kOk = 0;
constexpr int kErrInvalid = -1;
constexpr int kErrNoMem = -2;
constexpr int kErrCuda = -3;
constexpr int kErrTimeout = -4;
constexpr int kErrUnsupported = -5;
constexpr int kErrInternal = -6;

struct Options {
  int64_t pivot_rule = 0;
  int64_t small_cutoff = 2048;
  int64_t depth_limit = -1;
  int64_t timing = 0;
  int64_t tile_variant = 0;
  int64_t local_cutoff = 0;    // -1: the largest segment one block holds; 0: off
  int64_t wait_limit = int64_t(1) << 26;   // polls of a bounded device-side wait
  int64_t test_stall = 0;      // 1: the next sort's first partition launch stalls one tile
  int64_t level_loop = 0;      // 1: the host enqueues levels ahead instead of reading counts
  int64_t small_sort = 0;      // 1: 256-thread block networks for every small segment
  int64_t overlap = 0;         // 1: sorting networks on a second stream, beside the partitions
  int64_t local_sort = 0;      // leaves per segment the single-block local partitioning sorts
  int64_t coop_max = 0;        // single arrays up to this size: one cooperative launch (0: off)
};

struct Call {
  void* keys = nullptr;
  uint32_t* vals = nullptr;            // key-value sorts
  int64_t n = 0;                       // total keys
  const int64_t* seg_offsets = nullptr;
  int64_t nseg = 0;
  bool partition_only = false;         // bqs_partition
  void* out = nullptr;
  uint64_t pivot_raw = 0;
  int64_t* split = nullptr;
  void* stream = nullptr;
  Options opt;
  // Allocation-free calls only (bqs_sort_noalloc): a fixed device scratch area to use
  // instead of any allocation, and no pinned host buffer or timing events either.
  void* fixed_ws = nullptr;
  int64_t fixed_ws_bytes = 0;
};

struct Stats {
  int64_t levels = 0, partition_launches = 0, active_keys = 0, moved_keys = 0, equal_keys = 0;
  int64_t small_segments = 0, small_keys = 0, local_segments = 0, local_keys = 0;
  int64_t fallback_pivots = 0, kernel_launches = 0;
  double partition_ms = 0, partition_bytes_per_key = 0;
  double coop_ms = 0;   // duration of the cooperative launch (BQS_OPT_TIMING)
};

// Implemented in bqs_api.cu.
int fail_cuda(cudaError_t e, const char* what);
Options current_options();
void clear_stats();
int dispatch_call(int32_t dtype, const Call& c);   // runs c, keeps its statistics
int64_t layout_bytes(int64_t n, int key_size, bool pairs, int64_t nseg, int small_cutoff);
void user_workspace(void** ptr, int64_t* bytes);
void prepare_mempool();
// The calling thread's control-block readback buffer, two consecutive control blocks:
// pinned host memory the device can write (mapped = true), or pageable memory if
// pinning failed.
Ctrl* pinned_ctrl(bool* mapped);
std::vector<std::pair<cudaEvent_t, cudaEvent_t>>& timing_events();   // of the current device
// The calling thread's count events i = 0, 1 on the current device (null on failure).
cudaEvent_t counts_event(int i = 0);
// Deferred partition timing (BQS_OPT_TIMING = 2): an event pair the call may record and
// hand over with deferred_timing_push (work: the launch had tiles); bqs_timing_collect
// sums them.
int deferred_event_pair(cudaEvent_t* e0, cudaEvent_t* e1);
void deferred_timing_push(cudaEvent_t e0, cudaEvent_t e1, bool work);
// The calling thread's second stream and its eight events (i = 0..7) on the current
// device (null on failure): networks run there beside the partition levels
// (BQS_OPT_OVERLAP).
cudaStream_t side_stream();
cudaEvent_t side_event(int i);

// Implemented in the per-dtype translation units.
int run_i32(const Call& c, Stats& st);
int run_i64(const Call& c, Stats& st);
int run_f64(const Call& c, Stats& st);

}  // namespace bqs

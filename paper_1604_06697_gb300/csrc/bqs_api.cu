// C ABI of the BlockQuicksort library: argument checks, options, workspace, statistics,
// and dispatch to the per-dtype drivers.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <utility>
#include <vector>

#include "bqs.h"
#include "bqs_driver.cuh"
#include "bqs_internal.h"

namespace bqs {

namespace {
std::mutex g_opt_mu;
Options g_opt;
std::mutex g_ws_mu;
void* g_ws = nullptr;
int64_t g_ws_bytes = 0;
thread_local Stats t_stats;
thread_local char t_err[320];
thread_local Ctrl* t_pinned = nullptr;
// Events belong to the device that was current when they were created, so the
// per-thread caches are kept per device.
constexpr int kMaxDevices = 64;
thread_local std::vector<std::pair<cudaEvent_t, cudaEvent_t>> t_events[kMaxDevices];
thread_local cudaEvent_t t_counts_event[kMaxDevices][2];

int current_device_slot() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); dev = 0; }
  return dev >= 0 && dev < kMaxDevices ? dev : 0;
}

Options snapshot_options() {
  std::lock_guard<std::mutex> g(g_opt_mu);
  return g_opt;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

constexpr int64_t kMaxN = (int64_t)0xFFFFFFFFll;  // segment cursors hold 32-bit counts

int key_size(int32_t dtype) { return dtype == BQS_INT32 ? 4 : 8; }

int dispatch(int32_t dtype, const Call& c) {
  t_stats = Stats{};
  switch (dtype) {
    case BQS_INT32: return run_i32(c, t_stats);
    case BQS_INT64: return run_i64(c, t_stats);
    case BQS_FLOAT64: return run_f64(c, t_stats);
    default: return kErrInvalid;
  }
}
}  // namespace

Options current_options() { return snapshot_options(); }

void clear_stats() { t_stats = Stats{}; }

int dispatch_call(int32_t dtype, const Call& c) { return dispatch(dtype, c); }

int64_t layout_bytes(int64_t n, int key_size, bool pairs, int64_t nseg, int small_cutoff) {
  return (int64_t)plan_layout(n, key_size, pairs, nseg, small_cutoff, true).total;
}

int fail_cuda(cudaError_t e, const char* what) {
  std::snprintf(t_err, sizeof t_err, "CUDA error in %s: %s", what, cudaGetErrorString(e));
  cudaGetLastError();
  return kErrCuda;
}

void user_workspace(void** ptr, int64_t* bytes) {
  std::lock_guard<std::mutex> g(g_ws_mu);
  *ptr = g_ws;
  *bytes = g_ws_bytes;
}

// Keeps freed stream-ordered allocations in the device's default pool, so repeated
// calls do not return memory to the driver between sorts.
void prepare_mempool() {
  static std::mutex mu;
  static std::vector<int> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  std::lock_guard<std::mutex> g(mu);
  for (int d : done)
    if (d == dev) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
  done.push_back(dev);
}

Ctrl* pinned_ctrl(bool* mapped) {
  if (!t_pinned) {
    void* p = nullptr;
    if (cudaMallocHost(&p, 2 * sizeof(Ctrl)) != cudaSuccess) {
      cudaGetLastError();
      static thread_local Ctrl fallback[2];  // pageable: copies still complete on sync
      *mapped = false;
      return fallback;
    }
    t_pinned = (Ctrl*)p;
  }
  *mapped = true;
  return t_pinned;
}

std::vector<std::pair<cudaEvent_t, cudaEvent_t>>& timing_events() {
  return t_events[current_device_slot()];
}

thread_local cudaStream_t t_side_stream[kMaxDevices];
thread_local cudaEvent_t t_side_events[kMaxDevices][8];

cudaStream_t side_stream() {
  cudaStream_t& s = t_side_stream[current_device_slot()];
  if (!s && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    s = nullptr;
  }
  return s;
}

cudaEvent_t side_event(int i) {
  cudaEvent_t& e = t_side_events[current_device_slot()][i % 8];
  if (!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    e = nullptr;
  }
  return e;
}

// Deferred partition timing (BQS_OPT_TIMING = 2): event pairs of finished calls wait in
// `pending` until bqs_timing_collect; collected pairs return to `spare`.
struct DeferredTiming {
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> spare, pending;
  std::vector<char> work;
};
thread_local DeferredTiming t_deferred[kMaxDevices];

int deferred_event_pair(cudaEvent_t* e0, cudaEvent_t* e1) {
  DeferredTiming& d = t_deferred[current_device_slot()];
  if (d.spare.empty()) {
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return fail_cuda(e, "cudaEventCreate");
    e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
      cudaEventDestroy(a);
      return fail_cuda(e, "cudaEventCreate");
    }
    d.spare.emplace_back(a, b);
  }
  *e0 = d.spare.back().first;
  *e1 = d.spare.back().second;
  d.spare.pop_back();
  return kOk;
}

void deferred_timing_push(cudaEvent_t e0, cudaEvent_t e1, bool work) {
  DeferredTiming& d = t_deferred[current_device_slot()];
  d.pending.emplace_back(e0, e1);
  d.work.push_back(work ? 1 : 0);
}

cudaEvent_t counts_event(int i) {
  cudaEvent_t& e = t_counts_event[current_device_slot()][i & 1];
  if (!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    e = nullptr;
  }
  return e;
}

}  // namespace bqs

using namespace bqs;

extern "C" {

int bqs_sort(void* keys, int64_t n, int32_t dtype, bqs_stream_t stream) {
  if (dtype < BQS_INT32 || dtype > BQS_FLOAT64 || n < 0 || n > kMaxN) return BQS_ERR_INVALID;
  t_stats = Stats{};
  if (n <= 1) return BQS_OK;
  if (!keys || !aligned16(keys)) return BQS_ERR_INVALID;
  Call c;
  c.keys = keys;
  c.n = n;
  c.stream = stream;
  c.opt = snapshot_options();
  return dispatch(dtype, c);
}

int bqs_sort_pairs(void* keys, uint32_t* vals, int64_t n, int32_t dtype, bqs_stream_t stream) {
  if (dtype < BQS_INT32 || dtype > BQS_FLOAT64 || n < 0 || n > kMaxN) return BQS_ERR_INVALID;
  t_stats = Stats{};
  if (n <= 1) return BQS_OK;
  if (!keys || !vals || !aligned16(keys) || !aligned16(vals)) return BQS_ERR_INVALID;
  Call c;
  c.keys = keys;
  c.vals = vals;
  c.n = n;
  c.stream = stream;
  c.opt = snapshot_options();
  return dispatch(dtype, c);
}

int bqs_sort_segmented(void* keys, const int64_t* seg_offsets, int64_t nseg, int32_t dtype,
                       bqs_stream_t stream) {
  if (dtype < BQS_INT32 || dtype > BQS_FLOAT64 || nseg < 0) return BQS_ERR_INVALID;
  t_stats = Stats{};
  if (nseg == 0) return BQS_OK;
  if (!seg_offsets || ((uintptr_t)seg_offsets & 7u)) return BQS_ERR_INVALID;
  int64_t total = 0;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(&total, seg_offsets + nseg, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail_cuda(e, "reading seg_offsets[nseg]");
  if (total < 0 || total > kMaxN) return BQS_ERR_INVALID;
  if (total > 0 && (!keys || !aligned16(keys))) return BQS_ERR_INVALID;
  Call c;
  c.keys = keys;
  c.n = total;
  c.seg_offsets = seg_offsets;
  c.nseg = nseg;
  c.stream = stream;
  c.opt = snapshot_options();
  return dispatch(dtype, c);
}

int bqs_sort_batched(void* keys, int64_t n, const int64_t* seg_offsets, int64_t nseg,
                     int32_t dtype, bqs_stream_t stream) {
  if (dtype < BQS_INT32 || dtype > BQS_FLOAT64 || nseg < 0 || n < 0 || n > kMaxN)
    return BQS_ERR_INVALID;
  t_stats = Stats{};
  if (nseg == 0 || n == 0) return BQS_OK;
  if (!seg_offsets || ((uintptr_t)seg_offsets & 7u)) return BQS_ERR_INVALID;
  if (!keys || !aligned16(keys)) return BQS_ERR_INVALID;
  Call c;
  c.keys = keys;
  c.n = n;
  c.seg_offsets = seg_offsets;
  c.nseg = nseg;
  c.stream = stream;
  c.opt = snapshot_options();
  return dispatch(dtype, c);
}

int bqs_partition(const void* keys, int64_t n, const bqs_pivot* pivot, void* out, int64_t* split,
                  bqs_stream_t stream) {
  if (!pivot || !split || pivot->reserved != 0) return BQS_ERR_INVALID;
  const int32_t dtype = pivot->dtype;
  if (dtype < BQS_INT32 || dtype > BQS_FLOAT64 || n < 0 || n > kMaxN) return BQS_ERR_INVALID;
  t_stats = Stats{};
  if (n == 0) {
    *split = 0;
    return BQS_OK;
  }
  if (!keys || !out || !aligned16(keys) || !aligned16(out)) return BQS_ERR_INVALID;
  const uintptr_t a = (uintptr_t)keys, b = (uintptr_t)out, bytes = (uintptr_t)n * key_size(dtype);
  if (a < b + bytes && b < a + bytes) return BQS_ERR_INVALID;
  Call c;
  c.keys = (void*)keys;
  c.n = n;
  c.partition_only = true;
  c.out = out;
  c.split = split;
  c.stream = stream;
  c.opt = snapshot_options();
  if (dtype == BQS_INT32) c.pivot_raw = (uint32_t)pivot->v.i32;
  else if (dtype == BQS_INT64) c.pivot_raw = (uint64_t)pivot->v.i64;
  else std::memcpy(&c.pivot_raw, &pivot->v.f64, 8);
  return dispatch(dtype, c);
}

int bqs_set_option(int32_t opt, int64_t value) {
  std::lock_guard<std::mutex> g(g_opt_mu);
  switch (opt) {
    case BQS_OPT_PIVOT:
      if (value < 0 || value > 6) return BQS_ERR_INVALID;
      g_opt.pivot_rule = value;
      return BQS_OK;
    case BQS_OPT_SMALL_CUTOFF:
      if (value < 2 || value > kMaxSmallKeys) return BQS_ERR_INVALID;
      g_opt.small_cutoff = value;
      return BQS_OK;
    case BQS_OPT_DEPTH_LIMIT:
      if (value < -1 || value > 100000) return BQS_ERR_INVALID;
      g_opt.depth_limit = value;
      return BQS_OK;
    case BQS_OPT_TIMING:
      if (value < 0 || value > 2) return BQS_ERR_INVALID;
      g_opt.timing = value;
      return BQS_OK;
    case BQS_OPT_TILE:
      if (value < 0 || value > 5) return BQS_ERR_INVALID;  // the six variants() entries
      g_opt.tile_variant = value;
      return BQS_OK;
    case BQS_OPT_LOCAL_CUTOFF:
      if (value < -1 || value > (1 << 20)) return BQS_ERR_INVALID;
      g_opt.local_cutoff = value;
      return BQS_OK;
    case BQS_OPT_WAIT_LIMIT:
      if (value < 1 || value > 0xFFFFFFFFll) return BQS_ERR_INVALID;
      g_opt.wait_limit = value;
      return BQS_OK;
    case BQS_OPT_TEST_STALL:
      if (value < 0 || value > 1) return BQS_ERR_INVALID;
      g_opt.test_stall = value;
      return BQS_OK;
    case BQS_OPT_LEVEL_LOOP:
      if (value < 0 || value > 1) return BQS_ERR_INVALID;
      g_opt.level_loop = value;
      return BQS_OK;
    case BQS_OPT_SMALL_SORT:
      if (value < 0 || value > 1) return BQS_ERR_INVALID;
      g_opt.small_sort = value;
      return BQS_OK;
    case BQS_OPT_OVERLAP:
      if (value < 0 || value > 1) return BQS_ERR_INVALID;
      g_opt.overlap = value;
      return BQS_OK;
    case BQS_OPT_LOCAL_SORT:
      if (value < 0 || value > kLocalSortCap) return BQS_ERR_INVALID;
      g_opt.local_sort = value;
      return BQS_OK;
    case BQS_OPT_COOP_MAX:
      if (value < 0 || value > kMaxN) return BQS_ERR_INVALID;
      g_opt.coop_max = value;
      return BQS_OK;
    default:
      return BQS_ERR_UNSUPPORTED;
  }
}

int bqs_get_option(int32_t opt, int64_t* value) {
  if (!value) return BQS_ERR_INVALID;
  std::lock_guard<std::mutex> g(g_opt_mu);
  switch (opt) {
    case BQS_OPT_PIVOT: *value = g_opt.pivot_rule; return BQS_OK;
    case BQS_OPT_SMALL_CUTOFF: *value = g_opt.small_cutoff; return BQS_OK;
    case BQS_OPT_DEPTH_LIMIT: *value = g_opt.depth_limit; return BQS_OK;
    case BQS_OPT_TIMING: *value = g_opt.timing; return BQS_OK;
    case BQS_OPT_TILE: *value = g_opt.tile_variant; return BQS_OK;
    case BQS_OPT_LOCAL_CUTOFF: *value = g_opt.local_cutoff; return BQS_OK;
    case BQS_OPT_WAIT_LIMIT: *value = g_opt.wait_limit; return BQS_OK;
    case BQS_OPT_TEST_STALL: *value = g_opt.test_stall; return BQS_OK;
    case BQS_OPT_LEVEL_LOOP: *value = g_opt.level_loop; return BQS_OK;
    case BQS_OPT_SMALL_SORT: *value = g_opt.small_sort; return BQS_OK;
    case BQS_OPT_OVERLAP: *value = g_opt.overlap; return BQS_OK;
    case BQS_OPT_LOCAL_SORT: *value = g_opt.local_sort; return BQS_OK;
    case BQS_OPT_COOP_MAX: *value = g_opt.coop_max; return BQS_OK;
    default: return BQS_ERR_UNSUPPORTED;
  }
}

int bqs_workspace_bytes(int64_t n, int32_t dtype, int32_t with_payload, int64_t nseg,
                        int64_t* bytes) {
  if (!bytes || n < 0 || n > kMaxN || nseg < 0 || dtype < BQS_INT32 || dtype > BQS_FLOAT64)
    return BQS_ERR_INVALID;
  const Options o = snapshot_options();
  // A single array that may take the single-launch path also holds its end-of-launch
  // lists.
  const bool single_launch = with_payload == 0 && nseg == 0 && n <= o.coop_max &&
                             (uint64_t)n < kFusedMaxKeys;
  const Layout L = plan_layout(n, key_size(dtype), with_payload != 0, nseg, (int)o.small_cutoff, true,
                               single_launch);
  *bytes = (int64_t)L.total;
  return BQS_OK;
}

int bqs_set_workspace(void* ptr, int64_t bytes) {
  if (ptr && (bytes <= 0 || ((uintptr_t)ptr & 255u))) return BQS_ERR_INVALID;
  std::lock_guard<std::mutex> g(g_ws_mu);
  g_ws = ptr;
  g_ws_bytes = ptr ? bytes : 0;
  return BQS_OK;
}

int bqs_get_stats(bqs_stats* out) {
  if (!out) return BQS_ERR_INVALID;
  const Stats& s = t_stats;
  out->levels = s.levels;
  out->partition_launches = s.partition_launches;
  out->active_keys = s.active_keys;
  out->moved_keys = s.moved_keys;
  out->equal_keys = s.equal_keys;
  out->small_segments = s.small_segments;
  out->small_keys = s.small_keys;
  out->local_segments = s.local_segments;
  out->local_keys = s.local_keys;
  out->fallback_pivots = s.fallback_pivots;
  out->kernel_launches = s.kernel_launches;
  out->partition_ms = s.partition_ms;
  out->partition_bytes = (double)(s.active_keys + s.moved_keys) * s.partition_bytes_per_key;
  out->coop_ms = s.coop_ms;
  return BQS_OK;
}

int bqs_timing_collect(double* ms, int64_t* launches) {
  DeferredTiming& d = t_deferred[current_device_slot()];
  double total = 0;
  int64_t count = 0;
  int rc = BQS_OK;
  for (size_t i = 0; i < d.pending.size(); ++i) {
    if (rc == BQS_OK && d.work[i]) {
      cudaError_t e = cudaEventSynchronize(d.pending[i].second);
      float t = 0;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, d.pending[i].first, d.pending[i].second);
      if (e != cudaSuccess) rc = fail_cuda(e, "collecting partition timing");
      total += t;
      ++count;
    }
    d.spare.push_back(d.pending[i]);
  }
  d.pending.clear();
  d.work.clear();
  if (ms) *ms = total;
  if (launches) *launches = count;
  return rc;
}

const char* bqs_status_string(int status) {
  switch (status) {
    case BQS_OK: return "ok";
    case BQS_ERR_INVALID: return "invalid argument";
    case BQS_ERR_NOMEM: return "out of device memory for scratch";
    case BQS_ERR_CUDA: return t_err[0] ? t_err : "CUDA error";
    case BQS_ERR_TIMEOUT: return "device-side wait timed out";
    case BQS_ERR_UNSUPPORTED: return "unsupported option or combination";
    case kErrInternal: return "internal work list overflow";
    case BQS_ERR_TOO_LARGE:
      return "n exceeds the fixed scratch of bqs_sort_noalloc (at most 2^20 keys)";
    default: return "unknown status";
  }
}

}  // extern "C"

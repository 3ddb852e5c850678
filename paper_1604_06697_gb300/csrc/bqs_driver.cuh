// Host driver of the level-synchronous BlockQuicksort (one instantiation per key type).
//
// The Quicksort main loop of the paper (Sec. 2, Algorithm 1, with an explicit stack) is
// replaced by work lists processed breadth-first: every level partitions all unfinished
// large segments at once, and the children it produces are the next level's work.  The
// host only reads the next level's list counts (32 bytes) between levels.
#pragma once

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "bqs_coop.cuh"
#include "bqs_graph.cuh"
#include "bqs_internal.h"
#include "bqs_kernels.cuh"
#include "bqs_local.cuh"
#include "bqs_small.cuh"
#include "bqs_tma.cuh"

namespace bqs {

// ---- scratch layout ----------------------------------------------------------------------

struct Layout {
  size_t alt_key = 0, alt_val = 0, ctrl = 0;
  size_t tdone[2] = {0, 0};
  size_t large[2] = {0, 0}, cursor[2] = {0, 0}, small[2] = {0, 0}, tiny[2] = {0, 0}, todo[2] = {0, 0}, local[2] = {0, 0}, fill[2] = {0, 0}, group[2] = {0, 0}, big[2] = {0, 0};
  // Two more sets of network run lists (tiny, small, group, big) for sorts: the host
  // level loop rotates four sets, so that a level's bookkeeping waits only for the
  // networks of three levels before it.
  size_t spare_runs[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
  // Single-launch sort: the network runs and pivot-class fills of every level.
  size_t acc_runs = 0, acc_fill = 0;
  uint32_t cap_acc_runs = 0, cap_acc_fill = 0;
  size_t total = 0;
  uint32_t cap_large = 0, cap_run = 0, cap_fill = 0;
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Capacities: large segments are longer than the small cutoff and disjoint, so a level
// holds at most n/(C+1) of them; each yields at most two children (or, at the first
// level, one entry per caller segment).  Sized for C <= kMaxSmall, which holds for every
// sort that the cutoff applies to (key-value sorts clamp C to kMaxSmall).
inline Layout plan_layout(int64_t n, int key_size, bool pairs, int64_t nseg, int small_cutoff,
                          bool need_alt, bool single_launch = false) {
  Layout L;
  small_cutoff = std::min(small_cutoff, kMaxSmall);
  const uint64_t cap_large = (uint64_t)n / (uint64_t)(small_cutoff + 1) + 2;
  const uint64_t cap_run = std::max<uint64_t>(2 * cap_large, (uint64_t)nseg) + 2;
  L.cap_large = (uint32_t)std::min<uint64_t>(cap_large, 0xFFFFFFF0ull);
  L.cap_run = (uint32_t)std::min<uint64_t>(cap_run, 0xFFFFFFF0ull);
  L.cap_fill = L.cap_large;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes, 256); return at; };
  L.ctrl = take(sizeof(Ctrl));
  if (need_alt) {
    L.alt_key = take((size_t)n * key_size);
    if (pairs) L.alt_val = take((size_t)n * 4);
  }
  for (int i = 0; i < 2; ++i) {
    L.large[i] = take((size_t)L.cap_large * sizeof(Seg));
    L.cursor[i] = take((size_t)L.cap_large * 8);
    L.tdone[i] = take((size_t)L.cap_large * sizeof(unsigned long long));
    L.small[i] = take((size_t)L.cap_run * sizeof(Run));
    L.group[i] = take((size_t)L.cap_run * sizeof(Run));
    L.big[i] = take((size_t)L.cap_run * sizeof(Run));
    L.tiny[i] = take((size_t)L.cap_run * sizeof(Run));
    L.todo[i] = take((size_t)L.cap_large * sizeof(uint32_t));
    L.local[i] = take((size_t)L.cap_run * sizeof(Run));
    L.fill[i] = take((size_t)L.cap_fill * sizeof(Fill));
  }
  if (need_alt)
    for (int j = 0; j < 2; ++j)
      for (int k = 0; k < 4; ++k) L.spare_runs[j][k] = take((size_t)L.cap_run * sizeof(Run));
  if (single_launch) {
    // Every level appends at most two runs and one fill per large segment, at most
    // cap_large of them per level, over at most 2 log2 n + 3 + 8 key_size + 40 levels
    // (the default depth limit and one halving per key bit); never more runs or fills
    // than keys.  Past this the launch reports an overflow.
    int lg = 0;
    for (int64_t t = n; t > 1; t >>= 1) ++lg;
    const uint64_t levels = 2ull * (uint64_t)lg + 3 + 8ull * (uint64_t)key_size + 40;
    L.cap_acc_runs = (uint32_t)std::min<uint64_t>(std::min<uint64_t>((uint64_t)n, 2 * levels * cap_large) + 2,
                                                  0xFFFFFFF0ull);
    L.cap_acc_fill = (uint32_t)std::min<uint64_t>(std::min<uint64_t>((uint64_t)n, levels * cap_large) + 2,
                                                  0xFFFFFFF0ull);
    L.acc_runs = take((size_t)L.cap_acc_runs * sizeof(Run));
    L.acc_fill = take((size_t)L.cap_acc_fill * sizeof(Fill));
  }
  L.total = o;
  return L;
}

// Scratch for one call: the caller-set workspace when it fits, else stream-ordered
// allocation returned on the same stream.
struct Scratch {
  char* base = nullptr;
  bool owned = false;
  cudaStream_t st = nullptr;
  ~Scratch() {
    if (owned && base) cudaFreeAsync(base, st);
  }
};

inline int acquire_scratch(Scratch& s, size_t bytes, cudaStream_t st) {
  s.st = st;
  void* ws = nullptr;
  int64_t ws_bytes = 0;
  user_workspace(&ws, &ws_bytes);
  if (ws && (size_t)ws_bytes >= bytes) {
    s.base = (char*)ws;
    s.owned = false;
    return kOk;
  }
  prepare_mempool();
  void* p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, bytes, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? kErrNoMem : fail_cuda(e, "cudaMallocAsync");
  }
  s.base = (char*)p;
  s.owned = true;
  return kOk;
}

// ---- partition kernel variants -------------------------------------------------------------

struct Variant {
  int threads, kpt;
  const void* fn;
  size_t smem;        // dynamic shared memory per block
  // pdl: programmatic dependent launch (the blocks may start while the previous kernel
  // of the stream finishes; they wait for it before reading anything).
  void (*launch)(const Params&, int grid, cudaStream_t, bool pdl);
  void (*launch_fused)(const Params&, int grid, cudaStream_t, bool pdl);   // with the bookkeeping
  cudaError_t (*prepare)();  // allows its shared memory on the current device (before any use)
};

// A kernel that takes more than 48 KB of dynamic shared memory has to say so on every
// device it runs on: the attribute belongs to that device's context.  `devs` (one per
// kernel) remembers the devices on which it was set; a failed attribute call is
// returned (and tried again by the next call), and a device index outside 0..63 is
// refused rather than mistaken for another device.
inline cudaError_t allow_smem_on_device(const void* fn, size_t smem,
                                        std::atomic<unsigned long long>& devs) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  const unsigned long long bit = 1ull << dev;
  if (devs.load(std::memory_order_acquire) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  devs.fetch_or(bit, std::memory_order_acq_rel);
  return cudaSuccess;
}

template <class KT, bool PAIRS, int T, int K, int STAGES, int CHUNK, int MINB, bool FUSED>
void launch_partition_tma(const Params& P, int grid, cudaStream_t st, bool pdl) {
  const size_t smem = TmaShape<KT, PAIRS, T, K, STAGES, CHUNK>::smem;
  if (!pdl) {
    k_partition_tma<KT, PAIRS, T, K, STAGES, CHUNK, MINB, FUSED><<<grid, T, smem, st>>>(P);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)T);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_partition_tma<KT, PAIRS, T, K, STAGES, CHUNK, MINB, FUSED>, P);
}

template <class KT, bool PAIRS, int T, int K, int STAGES, int CHUNK, int MINB>
cudaError_t prepare_partition_tma() {
  static std::atomic<unsigned long long> devs{0}, devs_fused{0};
  const size_t smem = TmaShape<KT, PAIRS, T, K, STAGES, CHUNK>::smem;
  const cudaError_t e = allow_smem_on_device(
      (const void*)k_partition_tma<KT, PAIRS, T, K, STAGES, CHUNK, MINB, false>, smem, devs);
  if (e != cudaSuccess) return e;
  return allow_smem_on_device((const void*)k_partition_tma<KT, PAIRS, T, K, STAGES, CHUNK, MINB, true>,
                              smem, devs_fused);
}

template <class KT, bool PAIRS, int T, int K, int STAGES, int CHUNK = 256, int MINB = 1>
Variant make_tma_variant() {
  const void* fn = (const void*)k_partition_tma<KT, PAIRS, T, K, STAGES, CHUNK, MINB, false>;
  const size_t smem = TmaShape<KT, PAIRS, T, K, STAGES, CHUNK>::smem;
  return Variant{T, K, fn, smem, &launch_partition_tma<KT, PAIRS, T, K, STAGES, CHUNK, MINB, false>,
                 &launch_partition_tma<KT, PAIRS, T, K, STAGES, CHUNK, MINB, true>,
                 &prepare_partition_tma<KT, PAIRS, T, K, STAGES, CHUNK, MINB>};
}

// Tile shapes offered to the autotuner (BQS_OPT_TILE 0..4), all TMA-fed persistent
// kernels: keys per tile = threads * keys-per-thread, STAGES tiles in flight per block;
// 3 and 4 have smaller shared-memory footprints so that 3-4 blocks share an SM.
template <class KT, bool PAIRS>
const std::vector<Variant>& variants() {
  static const std::vector<Variant> v = [] {
    std::vector<Variant> r;
    if constexpr (sizeof(typename KT::U) == 4) {
      r.push_back(make_tma_variant<KT, PAIRS, 256, 16, 3>());
      r.push_back(make_tma_variant<KT, PAIRS, 256, 32, 2>());
      r.push_back(make_tma_variant<KT, PAIRS, 512, 16, 2>());
      r.push_back(make_tma_variant<KT, PAIRS, 256, 16, 2, 128>());
      r.push_back(make_tma_variant<KT, PAIRS, 256, 8, 4, 128>());
      r.push_back(make_tma_variant<KT, PAIRS, 256, 16, 2, 64, 4>());
    } else {
      r.push_back(make_tma_variant<KT, PAIRS, 256, 8, 3>());
      r.push_back(make_tma_variant<KT, PAIRS, 256, 16, 2>());
      r.push_back(make_tma_variant<KT, PAIRS, 512, 8, 2>());
      r.push_back(make_tma_variant<KT, PAIRS, 256, 8, 2, 128>());
      r.push_back(make_tma_variant<KT, PAIRS, 256, 4, 4, 128>());
      r.push_back(make_tma_variant<KT, PAIRS, 256, 8, 2, 64, 4>());
    }
    // Every variant on the first device at once; a failure here is returned by the
    // prepare() call that each sort makes for its own variant.
    for (const Variant& x : r) (void)x.prepare();
    cudaGetLastError();
    return r;
  }();
  return v;
}

// Shape of the single-block local partitioning: keys per block (L) and threads; both
// ping-pong buffers of L keys (+ payloads) fit in shared memory.  SORT: the block also
// sorts its finished sub-segments (key-only sorts).
template <class KT, bool PAIRS, bool SORT = false>
struct LocalCap {
  static constexpr int L = PAIRS ? 4096 : (int)(32768 / sizeof(typename KT::U));
  static constexpr int T = 256;
  static constexpr size_t smem = LocalShape<KT, PAIRS, L, T, SORT>::smem;
  static const void* fn() { return (const void*)k_local_partition<KT, PAIRS, L, T, SORT>; }
  // Allows the kernel's shared memory on the current device; called before its
  // occupancy is queried or it is launched there.
  static cudaError_t prepare() {
    static std::atomic<unsigned long long> devs{0};
    return allow_smem_on_device(fn(), smem, devs);
  }
  static int grid();
  static void launch(const Params& P, int p, int grid, cudaStream_t st) {
    k_local_partition<KT, PAIRS, L, T, SORT><<<grid, T, smem, st>>>(P, p);
  }
};

// Persistent grid of a kernel: resident blocks per SM times the SM count.
inline int persistent_grid(const void* fn, int threads, size_t smem) {
  static std::mutex mu;
  static std::vector<std::pair<const void*, int>> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> g(mu);
  for (auto& e : cache)
    if (e.first == fn) return e.second;
  int sms = 0, per = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem);
  const int g_ = std::max(1, sms * std::max(1, per));
  cache.emplace_back(fn, g_);
  return g_;
}

inline int sm_count() {
  static int sms = [] {
    int dev = 0, s = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
    return std::max(1, s);
  }();
  return sms;
}

template <class KT, bool PAIRS, bool SORT>
int LocalCap<KT, PAIRS, SORT>::grid() {
  return persistent_grid(fn(), T, smem);
}

// Allows the shared memory of the single-block local partitioning kernels that a call
// with these parameters may launch, on the current device.
template <class KT, bool PAIRS>
cudaError_t prepare_local(const Params& P) {
  if constexpr (!PAIRS) {
    if (P.local_sort) return LocalCap<KT, false, true>::prepare();
  }
  return LocalCap<KT, PAIRS, false>::prepare();
}

// Launches the single-block local partitioning over the `local` list of parity p:
// `count` runs when the host knows it (0: a persistent grid that reads it on the
// device); with P.local_sort the variant that sorts its finished sub-segments itself.
template <class KT, bool PAIRS>
void launch_local(const Params& P, int p, uint32_t count, cudaStream_t st) {
  if constexpr (!PAIRS) {
    if (P.local_sort) {
      using C = LocalCap<KT, false, true>;
      const int g = C::grid();
      C::launch(P, p, count ? (int)std::min<uint32_t>(count, (uint32_t)g) : g, st);
      return;
    }
  }
  using C = LocalCap<KT, PAIRS, false>;
  const int g = C::grid();
  C::launch(P, p, count ? (int)std::min<uint32_t>(count, (uint32_t)g) : g, st);
}

// ---- the level loop --------------------------------------------------------------------------

inline int status_code(int device_status) {
  if (device_status == kStatusInvalid) return kErrInvalid;
  if (device_status == kStatusTimeout) return kErrTimeout;
  return kErrInternal;
}

#define BQS_CK(call)                                              \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) return fail_cuda(e_, #call);           \
  } while (0)

// Non-blocking streams and events of the calling thread on the current device, used
// only to record the body of the device-side level loop into the conditional node's
// graph: the body forks onto the second stream (`fork`) and joins back (`join`).
struct BodyStreams {
  cudaStream_t hs = nullptr, hs2 = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  bool ok = false;
};

inline BodyStreams& body_streams() {
  static thread_local BodyStreams per_dev[64];   // streams and events belong to one device
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { cudaGetLastError(); dev = 0; }
  BodyStreams& b = per_dev[dev];
  if (!b.ok) {
    if ((!b.hs && cudaStreamCreateWithFlags(&b.hs, cudaStreamNonBlocking) != cudaSuccess) ||
        (!b.hs2 && cudaStreamCreateWithFlags(&b.hs2, cudaStreamNonBlocking) != cudaSuccess) ||
        (!b.fork && cudaEventCreateWithFlags(&b.fork, cudaEventDisableTiming) != cudaSuccess) ||
        (!b.join && cudaEventCreateWithFlags(&b.join, cudaEventDisableTiming) != cudaSuccess)) {
      cudaGetLastError();
      return b;
    }
    b.ok = true;
  }
  return b;
}

// Launches the sorting networks of the `small` list (kWarpSortMax+1 .. group_min keys)
// and of the `group` and `big` lists (longer segments, key-only sorts with
// small_sort = 0).  Key-only sorts: one warp per `small` segment (k_small_warps), one
// SmallGroup block per `group` segment (k_small_group) and per `big` segment
// (k_small_big, cutoffs above kMaxSmall); key-value sorts, or small_sort = 1: one
// 256-thread block per `small` segment (k_small_block), and `group` and `big` stay empty.
// Counts are the list lengths when the host knows them (a launch is then skipped when
// its list is empty); device_counts = true launches persistent grids that read them on
// the device.  Returns the number of launches.
template <class KT, bool PAIRS>
int launch_small(const Params& P, int p, uint32_t small, uint32_t group, uint32_t big,
                 bool device_counts, cudaStream_t s) {
  const int sms = sm_count();
  int n = 0;
  const bool warps = !PAIRS && P.small_sort == 0;
  if (device_counts || small) {
    if (warps) {
      const uint32_t g = device_counts ? 8 * sms : std::min<uint32_t>((small + 3) / 4, 8 * sms);
      if constexpr (!PAIRS) k_small_warps<KT, PAIRS><<<(int)g, 128, 0, s>>>(P, p);
    } else {
      const uint32_t g = device_counts ? 16 * sms : std::min<uint32_t>(small, 16 * sms);
      if constexpr (PAIRS) {
        if (P.small_sort == 0) {   // packable segments first; k_small_block takes the rest
          k_small_pairs_packed<KT><<<(int)g, 128, 0, s>>>(P, p);
          ++n;
        }
      }
      k_small_block<KT, PAIRS><<<(int)g, 256, 0, s>>>(P, p);
    }
    ++n;
  }
  if constexpr (!PAIRS) {
    if (warps && P.small_cutoff > P.group_min && (device_counts || group)) {
      const uint32_t g = device_counts ? 16 * sms : std::min<uint32_t>(group, 16 * sms);
      k_small_group<KT, PAIRS><<<(int)g, SmallGroup<KT>::T, 0, s>>>(P, p);
      ++n;
    }
    if (warps && P.small_cutoff > kMaxSmall && (device_counts || big)) {
      const uint32_t g = device_counts ? 8 * sms : std::min<uint32_t>(big, 8 * sms);
      k_small_big<KT, PAIRS><<<(int)g, SmallGroup<KT>::TBIG, 0, s>>>(P, p);
      ++n;
    }
  }
  return n;
}

// One level of the device-driven loop: every kernel takes the level parity and its work
// counts from the control block, so the grids are fixed (persistent) sizes.  A level
// of parity p has two independent parts:
//  * the partition part -- pivots, partition and children of the lists[p].large
//    segments (children go to lists[p ^ 1]), their pivot-class fills (lists[p].fill)
//    and the local partitioning of lists[p].local (leaves go to lists[p ^ 1]);
//  * the network part -- the segments that the previous level (or the initial split)
//    put on lists[p]'s tiny / small / group / big lists.
// They read disjoint lists and write disjoint key ranges, so they may run concurrently.
// Optional events bracket the partition launch for BQS_OPT_TIMING.
template <class KT, bool PAIRS>
void enqueue_level_partition(const Params& P, const Variant& var, cudaStream_t s, bool local_on,
                             cudaEvent_t e0, cudaEvent_t e1) {
  const int sms = sm_count();
  k_pivot<KT, PAIRS><<<8 * sms, 256, 0, s>>>(P);
  if (e0) cudaEventRecord(e0, s);
  var.launch(P, persistent_grid(var.fn, var.threads, var.smem), s, false);
  if (e1) cudaEventRecord(e1, s);
  k_bookkeep<KT, PAIRS><<<4 * sms, 256, 0, s>>>(P);
  k_fill<KT, PAIRS><<<4 * sms, 256, 0, s>>>(P, 0);
  if (local_on) launch_local<KT, PAIRS>(P, 0, 0, s);
}

template <class KT, bool PAIRS>
void enqueue_level_networks(const Params& P, cudaStream_t s) {
  k_small_warp<KT, PAIRS><<<16 * sm_count(), 256, 0, s>>>(P, 0);
  launch_small<KT, PAIRS>(P, 0, 0, 0, 0, true, s);
}

// Both parts in order on one stream.
template <class KT, bool PAIRS>
void enqueue_level_body(const Params& P, const Variant& var, cudaStream_t s, bool local_on,
                        cudaEvent_t e0, cudaEvent_t e1) {
  k_level_begin<<<1, 32, 0, s>>>(P);
  enqueue_level_partition<KT, PAIRS>(P, var, s, local_on, e0, e1);
  enqueue_level_networks<KT, PAIRS>(P, s);
}

// Pinned flags and events of the calling thread for the device-driven host loop.
struct LevelRing {
  int* flags = nullptr;            // pinned, 8 entries
  cudaEvent_t ev[8] = {};
  bool ok = false;
};

inline LevelRing& level_ring() {
  static thread_local LevelRing rings[64];   // per device: events belong to one device
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { cudaGetLastError(); dev = 0; }
  LevelRing& r = rings[dev];
  if (!r.ok) {
    void* p = nullptr;
    if (cudaMallocHost(&p, 8 * sizeof(int)) != cudaSuccess) { cudaGetLastError(); return r; }
    r.flags = (int*)p;
    for (auto& e : r.ev)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return r;
      }
    r.ok = true;
  }
  return r;
}

// Adds to the graph being captured on `s` a conditional while node whose body is one
// level of the sort, recorded on a helper stream with fixed (persistent) grids; the
// kernels read the level parity and the work counts from the control block, and
// k_level_end sets the loop condition.
template <class KT, bool PAIRS>
int capture_level_loop(const Params& P, const Variant& var, cudaStream_t s, int max_levels,
                       bool local_on) {
  cudaStreamCaptureStatus cs;
  unsigned long long id = 0;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edata = nullptr;
  size_t nd = 0;
  BQS_CK(cudaStreamGetCaptureInfo(s, &cs, &id, &g, &deps, &edata, &nd));
  cudaGraphConditionalHandle h;
  BQS_CK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  BQS_CK(cudaGraphAddNode(&node, g, deps, edata, nd, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  BQS_CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));

  BodyStreams& bs = body_streams();
  if (!bs.ok) return kErrCuda;
  cudaStream_t hs = bs.hs;
  BQS_CK(cudaStreamBeginCaptureToGraph(hs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  // The body forks after k_level_begin: the networks of the previous level's small
  // segments run on a parallel branch beside this level's partition part.
  k_level_begin<<<1, 32, 0, hs>>>(P);
  cudaEventRecord(bs.fork, hs);
  cudaStreamWaitEvent(bs.hs2, bs.fork, 0);
  enqueue_level_networks<KT, PAIRS>(P, bs.hs2);
  cudaEventRecord(bs.join, bs.hs2);
  enqueue_level_partition<KT, PAIRS>(P, var, hs, local_on, nullptr, nullptr);
  cudaStreamWaitEvent(hs, bs.join, 0);
  k_level_end<<<1, 32, 0, hs>>>(P, h, max_levels);
  const cudaError_t launch_err = cudaGetLastError();
  cudaGraph_t captured = nullptr;
  const cudaError_t end_err = cudaStreamEndCapture(hs, &captured);
  if (launch_err != cudaSuccess) return fail_cuda(launch_err, "recording the level loop");
  if (end_err != cudaSuccess) return fail_cuda(end_err, "cudaStreamEndCapture(level loop body)");
  return kOk;
}

// The level loop driven by device-side counts on an ordinary stream: the host keeps up
// to kAhead levels enqueued and, before adding level j + kAhead, waits for level j's
// flag (copied to pinned memory behind an event).  Levels enqueued past the last one
// find empty lists and return at once.  Returns after the last level has run.
// Copies the control block to the host.  Into pinned (device-mapped) memory a one-block
// kernel writes it directly: a DMA copy would queue behind any large transfer the
// caller has on the same copy engine (an upload or download overlapping the sort).
static __global__ void k_ctrl_to_host(const Ctrl* __restrict__ c, Ctrl* h) {
  static_assert(sizeof(Ctrl) % 8 == 0, "control block in 8-byte words");
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(c);
  unsigned long long* dst = reinterpret_cast<unsigned long long*>(h);
  for (int i = threadIdx.x; i < (int)(sizeof(Ctrl) / 8); i += blockDim.x) dst[i] = src[i];
}

inline cudaError_t read_ctrl(const Ctrl* dev, Ctrl* host, bool mapped, cudaStream_t s) {
  if (!mapped) return cudaMemcpyAsync(host, dev, sizeof(Ctrl), cudaMemcpyDeviceToHost, s);
  k_ctrl_to_host<<<1, 64, 0, s>>>(dev, host);
  return cudaGetLastError();
}

template <class KT, bool PAIRS>
int run_levels_ahead(Params P, const Variant& var, cudaStream_t s, int max_levels,
                     bool local_on, bool timing, int test_stall, Ctrl* host, bool host_mapped,
                     Stats& st) {
  constexpr int kAhead = 4;   // < 8, the size of the flag ring
  LevelRing& ring = level_ring();
  if (!ring.ok) return kErrNoMem;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>>& evs = timing_events();
  std::vector<char> partitioned;
  int enq = 0, checked = 0;
  for (bool more = true; more;) {
    for (; enq < checked + kAhead && enq <= max_levels; ++enq) {
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (timing) {
        if ((size_t)enq == evs.size()) {
          cudaEvent_t a, b;
          BQS_CK(cudaEventCreate(&a));
          BQS_CK(cudaEventCreate(&b));
          evs.emplace_back(a, b);
        }
        e0 = evs[enq].first; e1 = evs[enq].second;
      }
      P.test_stall = enq == 0 ? test_stall : 0;
      enqueue_level_body<KT, PAIRS>(P, var, s, local_on, e0, e1);
      k_level_step<<<1, 32, 0, s>>>(P, max_levels);
      BQS_CK(cudaGetLastError());
      BQS_CK(cudaMemcpyAsync(&ring.flags[enq & 7], &P.ctrl->more[enq & 7], sizeof(int),
                             cudaMemcpyDeviceToHost, s));
      BQS_CK(cudaEventRecord(ring.ev[enq & 7], s));
      st.kernel_launches += (local_on ? 8 : 7) +
                            ((!PAIRS && P.small_sort == 0 && P.small_cutoff > P.group_min) ? 2 : 1) +
                            ((!PAIRS && P.small_sort == 0 && P.small_cutoff > kMaxSmall) ? 1 : 0);
      st.partition_launches += 1;
    }
    if (checked == enq) return kErrInternal;   // the device bounds the levels first
    BQS_CK(cudaEventSynchronize(ring.ev[checked & 7]));
    const int f = *(volatile int*)&ring.flags[checked & 7];
    partitioned.push_back((f & 2) != 0);
    more = (f & 1) != 0;
    ++checked;
  }
  BQS_CK(read_ctrl(P.ctrl, host, host_mapped, s));
  BQS_CK(cudaStreamSynchronize(s));
  if (host->status) return status_code(host->status);
  st.levels = (int64_t)host->levels_run;
  st.active_keys = (int64_t)host->active_total;
  st.local_segments = (int64_t)host->local_runs;
  st.small_segments = (int64_t)host->acc.small;
  st.moved_keys = (int64_t)host->moved_keys;
  st.equal_keys = (int64_t)host->equal_keys;
  st.small_keys = (int64_t)host->small_keys;
  st.local_keys = (int64_t)host->local_keys;
  st.fallback_pivots = (int64_t)host->fallbacks;
  st.partition_bytes_per_key = (double)sizeof(typename KT::U) + (PAIRS ? 4.0 : 0.0);
  if (timing) {
    double ms = 0;
    for (size_t i = 0; i < partitioned.size(); ++i) {
      if (!partitioned[i]) continue;
      float t = 0;
      BQS_CK(cudaEventElapsedTime(&t, evs[i].first, evs[i].second));
      ms += t;
    }
    st.partition_ms = ms;
  }
  return kOk;
}

// The single-launch sort (bqs_coop.cuh): one cooperative launch over a persistent grid,
// then one read-back of the control block.  Returns kCoopRefused (nothing enqueued)
// when the device cannot make every block resident; the caller then runs the host loop.
constexpr int kCoopRefused = 1;

template <class KT>
int run_coop(Params P, int64_t n, int max_levels, bool timing, int test_stall, cudaStream_t s,
             Ctrl* host, bool host_mapped, Stats& st, Run* acc_runs, uint32_t cap_acc_runs,
             Fill* acc_fill, uint32_t cap_acc_fill) {
  const void* fn = (const void*)k_coop_sort<KT>;
  const int grid = persistent_grid(fn, kCoopThreads, CoopShape<KT>::smem);
  int coop = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) {
    cudaGetLastError();
    return kCoopRefused;
  }
  P.local_cutoff = P.small_cutoff;   // no single-block local partitioning here
  P.tile = CoopShape<KT>::TILE;      // the tile space of this kernel's partition step
  // Network runs of every size and pivot-class fills go to one list each, kept for the
  // end of the launch.
  P.net_acc = &P.ctrl->acc;
  for (int i = 0; i < 2; ++i) {
    P.l.tiny[i] = P.l.small[i] = P.l.group[i] = P.l.big[i] = acc_runs;
    P.l.fill[i] = acc_fill;
  }
  P.l.cap_run = cap_acc_runs;
  P.l.cap_fill = cap_acc_fill;
  P.test_stall = test_stall;
  P.device_loop = 0;
  void* args[] = {(void*)&P, (void*)&n, (void*)&max_levels};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (timing) {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>>& evs = timing_events();
    if (evs.empty()) {
      cudaEvent_t a, b;
      BQS_CK(cudaEventCreate(&a));
      BQS_CK(cudaEventCreate(&b));
      evs.emplace_back(a, b);
    }
    e0 = evs[0].first;
    e1 = evs[0].second;
    BQS_CK(cudaEventRecord(e0, s));
  }
  const cudaError_t le = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kCoopThreads), args,
                                                     CoopShape<KT>::smem, s);
  if (le == cudaErrorCooperativeLaunchTooLarge) {
    cudaGetLastError();
    return kCoopRefused;
  }
  if (le != cudaSuccess) return fail_cuda(le, "cudaLaunchCooperativeKernel(k_coop_sort)");
  if (timing) BQS_CK(cudaEventRecord(e1, s));
  BQS_CK(read_ctrl(P.ctrl, host, host_mapped, s));
  BQS_CK(cudaStreamSynchronize(s));
  if (host->status) return status_code(host->status);
  st.kernel_launches += 2;   // the sort and the control-block read-back
  st.levels = (int64_t)host->levels_run;
  st.partition_launches = 0;
  st.active_keys = (int64_t)host->active_total;
  st.moved_keys = (int64_t)host->moved_keys;
  st.equal_keys = (int64_t)host->equal_keys;
  st.small_keys = (int64_t)host->small_keys;
  st.small_segments = (int64_t)host->acc.small;
  st.fallback_pivots = (int64_t)host->fallbacks;
  st.partition_bytes_per_key = (double)sizeof(typename KT::U);
  if (timing) {
    float ms = 0;
    BQS_CK(cudaEventElapsedTime(&ms, e0, e1));
    st.coop_ms = ms;
  }
  return kOk;
}

template <class KT, bool PAIRS>
int run_call(const Call& c, Stats& st) {
  using U = typename KT::U;
  const cudaStream_t s = (cudaStream_t)c.stream;
  const auto& vars = variants<KT, PAIRS>();
  const Variant& var = vars[(size_t)std::min<int64_t>(std::max<int64_t>(c.opt.tile_variant, 0), (int64_t)vars.size() - 1)];
  {   // before its occupancy query and every launch path below
    const cudaError_t e = var.prepare();
    if (e != cudaSuccess) return fail_cuda(e, "cudaFuncSetAttribute (partition kernel)");
  }
  const int tile = var.threads * var.kpt;
  // Cutoffs above kMaxSmall apply to key-only sorts with the warp-group networks.
  const int small_cutoff = c.partition_only ? 1
                           : (PAIRS || c.opt.small_sort) ? (int)std::min<int64_t>(c.opt.small_cutoff, kMaxSmall)
                                                         : (int)c.opt.small_cutoff;
  // Segments up to local_cutoff keys are partitioned down to the small-segment cutoff by
  // one thread block in shared memory (not below a cutoff of kWarpSortMax keys: the
  // block's sub-segment lists are sized for that).
  constexpr int kLocalL = LocalCap<KT, PAIRS>::L;
  const int local_cutoff =
      (c.partition_only || small_cutoff < kWarpSortMax)
          ? small_cutoff
          : std::max(small_cutoff, c.opt.local_cutoff < 0
                                       ? kLocalL
                                       : (int)std::min<int64_t>(c.opt.local_cutoff, kLocalL));

  // Single arrays of up to BQS_OPT_COOP_MAX keys (fewer than kFusedMaxKeys) may run
  // every level in one launch.
  const bool single_launch = !PAIRS && !c.fixed_ws && !c.partition_only && !c.seg_offsets &&
                             c.opt.level_loop == 0 && c.opt.small_sort == 0 &&
                             local_cutoff <= small_cutoff && c.n > small_cutoff &&
                             c.n <= c.opt.coop_max && (uint64_t)c.n < kFusedMaxKeys;
  const Layout L = plan_layout(c.n, (int)sizeof(U), PAIRS, c.nseg, small_cutoff, !c.partition_only,
                               single_launch);
  Scratch scratch;
  int rc = kOk;
  if (c.fixed_ws) {   // allocation-free call: the caller's fixed scratch must be enough
    if ((size_t)c.fixed_ws_bytes < L.total) return kErrInvalid;
    scratch.base = (char*)c.fixed_ws;
  } else {
    rc = acquire_scratch(scratch, L.total, s);
  }
  if (rc) return rc;
  char* w = scratch.base;

  Params P{};
  P.ctrl = (Ctrl*)(w + L.ctrl);
  if (c.partition_only) {
    P.b.key[0] = c.keys; P.b.key[1] = c.out; P.b.final_key = c.out;
  } else {
    P.b.key[0] = c.keys; P.b.key[1] = w + L.alt_key; P.b.final_key = c.keys;
    if (PAIRS) {
      P.b.val[0] = c.vals; P.b.val[1] = (uint32_t*)(w + L.alt_val); P.b.final_val = c.vals;
    }
  }
  for (int i = 0; i < 2; ++i) {
    P.l.large[i] = (Seg*)(w + L.large[i]);
    P.l.cursor[i] = (unsigned long long*)(w + L.cursor[i]);
    P.l.tdone[i] = (unsigned long long*)(w + L.tdone[i]);
    P.l.small[i] = (Run*)(w + L.small[i]);
    P.l.group[i] = (Run*)(w + L.group[i]);
    P.l.big[i] = (Run*)(w + L.big[i]);
    P.l.tiny[i] = (Run*)(w + L.tiny[i]);
    P.l.todo[i] = (uint32_t*)(w + L.todo[i]);
    P.l.local[i] = (Run*)(w + L.local[i]);
    P.l.fill[i] = (Fill*)(w + L.fill[i]);
  }
  P.l.cap_large = L.cap_large; P.l.cap_run = L.cap_run; P.l.cap_fill = L.cap_fill;
  P.pivot_rule = c.opt.pivot_rule;
  P.small_cutoff = small_cutoff;
  P.local_cutoff = local_cutoff;
  P.route_children = c.partition_only ? 0 : 1;
  P.tile = tile;
  P.n_keys = c.n;
  P.wait_limit = (uint32_t)c.opt.wait_limit;
  P.test_stall = 0;
  P.small_sort = (int)c.opt.small_sort;
  P.local_sort = (!PAIRS && P.small_sort == 0) ? (int)c.opt.local_sort : 0;
  // Small segments above one warp's capacity go to the `group` list (key-only sorts with
  // the warp networks); otherwise every small segment above kWarpSortMax is `small`.
  P.group_min = (!PAIRS && P.small_sort == 0) ? small_warp_max<KT, PAIRS>() : kMaxSmall;
  {
    int64_t top = c.n;  // depth limit 2*floor(log2 n)+3 of the largest array (Sec. 2)
    int lg = 0;
    while (top > 1) { top >>= 1; ++lg; }
    P.depth_limit = c.opt.depth_limit >= 0 ? (int)c.opt.depth_limit : 2 * lg + 3;
  }
  if (local_cutoff > small_cutoff) {
    const cudaError_t e = prepare_local<KT, PAIRS>(P);
    if (e != cudaSuccess) return fail_cuda(e, "cudaFuncSetAttribute (local partitioning)");
  }

  // On a stream that is being captured into a CUDA graph the level loop runs on the
  // device (nothing can be read back while capturing).
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  BQS_CK(cudaStreamIsCapturing(s, &cap));
  const bool device_loop = cap == cudaStreamCaptureStatusActive && !c.fixed_ws;
  if (device_loop && c.partition_only) return kErrUnsupported;   // split is read back
  if (!device_loop && !c.fixed_ws) body_streams();   // created outside any capture

  static thread_local Ctrl pageable_ctrl;
  bool host_mapped = false;
  Ctrl* host = (c.fixed_ws || device_loop) ? &pageable_ctrl : pinned_ctrl(&host_mapped);
  const bool timing = c.opt.timing && !c.fixed_ws && !device_loop;
  BQS_CK(cudaMemsetAsync(P.ctrl, 0, sizeof(Ctrl), s));

  if constexpr (!PAIRS) {
    // Single arrays of up to BQS_OPT_COOP_MAX keys: every level in one launch.
    if (!device_loop && single_launch) {
      const int rc_coop = run_coop<KT>(P, c.n, P.depth_limit + 8 * (int)sizeof(U) + 40, timing,
                                       c.opt.test_stall ? 1 : 0, s, host, host_mapped, st,
                                       (Run*)(w + L.acc_runs), L.cap_acc_runs,
                                       (Fill*)(w + L.acc_fill), L.cap_acc_fill);
      if (rc_coop != kCoopRefused) return rc_coop;
    }
  }

  ListCounts cur{};
  bool host_fresh = false;   // `host` holds this call's control block
  if (device_loop) {
    if (c.seg_offsets) {
      const int g = (int)std::min<int64_t>((c.nseg + 255) / 256, 4 * sm_count());
      k_init_segments<KT, PAIRS><<<g, 256, 0, s>>>(P, c.seg_offsets, c.nseg);
    } else {
      k_init_single<KT, PAIRS><<<1, 32, 0, s>>>(P, c.n);
    }
    BQS_CK(cudaGetLastError());
    const int max_levels = P.depth_limit + 8 * (int)sizeof(U) + 40;
    P.device_loop = 1;
    P.p = 0;
    st.kernel_launches += 10;   // per level
    return capture_level_loop<KT, PAIRS>(P, var, s, max_levels, local_cutoff > small_cutoff);
  } else if (!c.fixed_ws && !c.partition_only && c.opt.level_loop == 1) {
    if (c.seg_offsets) {
      const int g = (int)std::min<int64_t>((c.nseg + 255) / 256, 4 * sm_count());
      k_init_segments<KT, PAIRS><<<g, 256, 0, s>>>(P, c.seg_offsets, c.nseg);
    } else {
      k_init_single<KT, PAIRS><<<1, 32, 0, s>>>(P, c.n);
    }
    st.kernel_launches += 1;
    BQS_CK(cudaGetLastError());
    const int max_levels = P.depth_limit + 8 * (int)sizeof(U) + 40;
    P.device_loop = 1;
    P.p = 0;
    return run_levels_ahead<KT, PAIRS>(P, var, s, max_levels, local_cutoff > small_cutoff, timing,
                                       c.opt.test_stall ? 1 : 0, host, host_mapped, st);
  } else if (c.partition_only) {
    k_init_partition<KT><<<1, 32, 0, s>>>(P, c.n, c.pivot_raw);
    st.kernel_launches += 1;
    cur.large = 1ull | ((unsigned long long)((c.n - 1) / tile + 1) << 32);
    cur.large_keys = (unsigned long long)c.n;
  } else if (c.seg_offsets) {
    const int g = (int)std::min<int64_t>((c.nseg + 255) / 256, 4 * sm_count());
    k_init_segments<KT, PAIRS><<<g, 256, 0, s>>>(P, c.seg_offsets, c.nseg);
    st.kernel_launches += 1;
    BQS_CK(cudaGetLastError());
    BQS_CK(read_ctrl(P.ctrl, host, host_mapped, s));
    BQS_CK(cudaStreamSynchronize(s));
    if (host->status) return status_code(host->status);
    cur = host->lists[0];
    host_fresh = true;
  } else {
    k_init_single<KT, PAIRS><<<1, 32, 0, s>>>(P, c.n);
    st.kernel_launches += 1;
    if (c.n <= small_cutoff && c.n <= kWarpSortMax) cur.tiny = 1;
    else if (c.n <= small_cutoff && c.n > kMaxSmall) cur.big = 1;
    else if (c.n <= small_cutoff && c.n > P.group_min) cur.group = 1;
    else if (c.n <= small_cutoff) cur.small = 1;
    else if (c.n <= local_cutoff) cur.local = 1;
    else {
      cur.large = 1ull | ((unsigned long long)((c.n - 1) / tile + 1) << 32);
      cur.large_keys = (unsigned long long)c.n;
      // mirrors inline_pivot(): which first segments leave their pivot to k_pivot
      cur.todo = (P.depth_limit <= 0 || (P.pivot_rule == 1 && c.n >= 20000)) ? 1 : 0;
    }
  }
  BQS_CK(cudaGetLastError());

  const int sms = sm_count();
  const int part_grid_max = persistent_grid(var.fn, var.threads, var.smem);
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>>& evs = timing_events();
  size_t ev_used = 0;

  // Every level removes the pivot class of each segment, and past the depth limit the
  // range-midpoint pivot halves the key range: more levels than this means a bug.
  const int max_levels = P.depth_limit + 8 * (int)sizeof(U) + 40;
  // Sorts read each level's counts behind an event right after its bookkeeping;
  // partitions and the allocation-free entry point (which creates no CUDA objects)
  // synchronise the stream at the end of each level instead.
  const cudaEvent_t counts_ev = (c.partition_only || c.fixed_ws) ? nullptr : counts_event();

  if (counts_ev && !c.partition_only) {
    // ---- the level loop with one level of lookahead ----------------------------------
    // The pivot pass and the partition kernel read their work counts from the control
    // block, so level L+1's are enqueued (fixed grids) right after level L's bookkeeping
    // and count read-back, before the host waits for those counts: the device never
    // idles while the host turns around.  Networks (of the lists of parity p, written by
    // the previous bookkeeping) run beside the partitions on a second stream with
    // BQS_OPT_OVERLAP.  Their run lists rotate over four sets: level L's networks read
    // set L mod 4, which the bookkeeping of level L-1 wrote, and level L's bookkeeping
    // writes set (L+1) mod 4, so it waits only for the networks of level L-3, which
    // read that set (`done[set]` marks the end of the networks that read a set).
    // `ready[set]` marks the end of the bookkeeping (and single-block partitioning)
    // that wrote a set.
    //
    // Without single-block partitioning, and with the control block in host-mapped
    // memory, the loop runs one level deeper: level L+1's bookkeeping is enqueued with
    // its partition, before the host has read level L's counts.  Its grid is sized for
    // twice level L's large segments (each has at most two large children; the kernel
    // reads the exact count on the device), and its last block copies the control block
    // into the other of two host-mapped blocks, behind the other of two events.
    cudaStream_t s1 = nullptr;
    constexpr int kSets = 4;
    cudaEvent_t ready[kSets] = {}, done[kSets] = {};
    if (c.opt.overlap) {
      s1 = side_stream();
      for (int k = 0; k < kSets; ++k) {
        ready[k] = side_event(k);
        done[k] = side_event(kSets + k);
        if (!ready[k] || !done[k]) s1 = nullptr;
      }
    }
    const cudaEvent_t counts_ev2 = counts_event(1);
    const bool deep = local_cutoff <= small_cutoff && host_mapped && counts_ev2 != nullptr;
    const cudaEvent_t cev[2] = {counts_ev, counts_ev2};
    Ctrl* const hbuf[2] = {host, host + 1};   // pinned_ctrl: two control blocks
    // Set 0 and 1 are the lists of parity 0 and 1 (the first level's runs, written
    // before the loop, are set 0); set 2 is the layout's spare set.
    Run* run_sets[kSets][4] = {{P.l.tiny[0], P.l.small[0], P.l.group[0], P.l.big[0]},
                               {P.l.tiny[1], P.l.small[1], P.l.group[1], P.l.big[1]},
                               {(Run*)(w + L.spare_runs[0][0]), (Run*)(w + L.spare_runs[0][1]),
                                (Run*)(w + L.spare_runs[0][2]), (Run*)(w + L.spare_runs[0][3])},
                               {(Run*)(w + L.spare_runs[1][0]), (Run*)(w + L.spare_runs[1][1]),
                                (Run*)(w + L.spare_runs[1][2]), (Run*)(w + L.spare_runs[1][3])}};
    auto with_runs = [&](Params X, int parity, int set) {
      X.l.tiny[parity] = run_sets[set][0];
      X.l.small[parity] = run_sets[set][1];
      X.l.group[parity] = run_sets[set][2];
      X.l.big[parity] = run_sets[set][3];
      return X;
    };
    bool side_work[kSets] = {};
    auto join = [&]() {
      for (int k = 0; k < kSets; ++k)
        if (side_work[k]) cudaStreamWaitEvent(s, done[k], 0);
    };
    struct Join {
      decltype(join)& f;
      ~Join() { f(); }
    } join_on_exit{join};
    std::vector<char> timed_work;   // per timed partition launch: whether it had tiles
    // BQS_OPT_TIMING = 2: each launch gets its own event pair, handed over at the end of
    // the call for bqs_timing_collect, and the call never waits for them.
    const bool deferred = timing && c.opt.timing == 2;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> call_evs;
    // X: the launch's parameters when they differ from P, with the fused bookkeeping.
    auto launch_partition = [&](int p, int grid, int stall, const Params* X = nullptr) -> int {
      P.p = p;
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (deferred) {
        const int erc = deferred_event_pair(&e0, &e1);
        if (erc) return erc;
        call_evs.emplace_back(e0, e1);
        BQS_CK(cudaEventRecord(e0, s));
      } else if (timing) {
        if (ev_used == evs.size()) {
          cudaEvent_t a, b;
          BQS_CK(cudaEventCreate(&a));
          BQS_CK(cudaEventCreate(&b));
          evs.emplace_back(a, b);
        }
        e0 = evs[ev_used].first;
        e1 = evs[ev_used].second;
        ++ev_used;
        BQS_CK(cudaEventRecord(e0, s));
      }
      Params Y = X ? *X : P;
      Y.p = p;
      Y.test_stall = stall;
      (X ? var.launch_fused : var.launch)(Y, grid, s, deep);
      if (timing) BQS_CK(cudaEventRecord(e1, s));
      st.kernel_launches += 1;
      return kOk;
    };
    // Every way out of the call hands the deferred pairs over (their recorded launches
    // will complete; one whose outcome is unknown counts as having had work).
    struct HandOver {
      std::vector<std::pair<cudaEvent_t, cudaEvent_t>>& evs;
      std::vector<char>& work;
      ~HandOver() {
        for (size_t i = 0; i < evs.size(); ++i)
          deferred_timing_push(evs[i].first, evs[i].second, i < work.size() ? work[i] != 0 : true);
      }
    } hand_over{call_evs, timed_work};
    // Bookkeeping of level lv (writes run set (lv+1) mod 3, waiting for the networks
    // that read it), sized for `bound` large segments; copy_to: where its last block
    // copies the control block (null: no copy).
    auto enqueue_bookkeep = [&](int lv, uint32_t bound, Ctrl* copy_to) -> int {
      const int bp = lv & 1, ws = (lv + 1) % kSets;
      if (side_work[ws]) BQS_CK(cudaStreamWaitEvent(s, done[ws], 0));
      Params B = with_runs(P, bp ^ 1, ws);
      B.p = bp;
      B.ctrl_host = copy_to;
      k_bookkeep<KT, PAIRS><<<(int)std::min<uint32_t>((bound + 255) / 256, 4 * sms), 256, 0, s>>>(B);
      st.kernel_launches += 1;
      return kOk;
    };
    // The deep loop can leave the call with one bookkeeping still to copy into the
    // thread's host-mapped blocks (the last level's, or after an error): every way out
    // waits for it, so that the next call does not read a block that is still written.
    struct LastCopy {
      cudaEvent_t ev = nullptr;
      ~LastCopy() {
        if (ev) cudaEventSynchronize(ev);
      }
    } last_copy;
    // Grids of the lookahead launches for the level after one with counts `lc`: its
    // segments are the large children of that level's, so at most 2 * lc.large of them,
    // holding at most lc.large_keys keys in at most large_keys / tile + 2 tiles each.
    // Both kernels take their work from the device and accept any grid; a small one
    // spares a deep level the launch of a full persistent grid.  (Without this bound
    // when the single-block partitioning can add work.)
    auto next_part_grid = [&](const ListCounts& lc) -> int {
      if (local_cutoff > small_cutoff) return part_grid_max;
      const uint64_t t = lc.large_keys / (uint64_t)tile + 4ull * (uint32_t)lc.large + 1;
      return (int)std::min<uint64_t>(t, (uint64_t)part_grid_max);
    };
    auto next_pivot_grid = [&](const ListCounts& lc) -> int {
      if (local_cutoff > small_cutoff) return 8 * sms;
      return (int)std::min<uint64_t>(2ull * (uint32_t)lc.large + 1, 8ull * sms);
    };
    // Levels of at most two tiles and two segments per partition block (deep loop only)
    // get the bookkeeping fused into the partition kernel: no bookkeeping launch, and
    // the counts are copied out by the block that finishes the level's last segment.
    // The lists a fused level appends to must be empty when it starts: a fused level
    // leaves its own consumed lists empty, the host clears them after any other level.
    bool prev_fused = true;   // lists[1] start empty (the control block was zeroed)
    // (Also fewer than kFusedMaxKeys keys: the fields of a segment's completion word.)
    auto fuse_ok = [&](uint64_t tiles_bound, uint64_t segs_bound, uint64_t keys_bound) {
      return deep && tiles_bound <= 2ull * (uint64_t)part_grid_max &&
             segs_bound <= 2ull * (uint64_t)part_grid_max && keys_bound < kFusedMaxKeys;
    };
    auto enqueue_fused_partition = [&](int lv, int grid, int stall) -> int {
      const int lp = lv & 1, ws = (lv + 1) % kSets;
      if (!prev_fused) BQS_CK(cudaMemsetAsync(&P.ctrl->lists[lp ^ 1], 0, sizeof(ListCounts), s));
      if (side_work[ws]) BQS_CK(cudaStreamWaitEvent(s, done[ws], 0));
      Params X = with_runs(P, lp ^ 1, ws);
      X.ctrl_host = hbuf[lp];
      return launch_partition(lp, grid, stall, &X);
    };
    if (s1) BQS_CK(cudaEventRecord(ready[0], s));   // the first lists' runs are written
    if ((uint32_t)cur.large) {   // level 0 from the host's own counts
      P.p = 0;
      if (cur.todo) {
        k_pivot<KT, PAIRS><<<(int)std::min<uint32_t>(cur.todo, 8 * sms), 256, 0, s>>>(P);
        st.kernel_launches += 1;
      }
      const uint32_t tiles0 = (uint32_t)(cur.large >> 32);
      const int grid0 = (int)std::min<uint32_t>(tiles0, (uint32_t)part_grid_max);
      const int stall0 = c.opt.test_stall ? 1 : 0;
      const bool fused0 = fuse_ok(tiles0, (uint32_t)cur.large, cur.large_keys);
      rc = fused0 ? enqueue_fused_partition(0, grid0, stall0) : launch_partition(0, grid0, stall0);
      if (rc) return rc;
      if (timing) timed_work.push_back(1);
      prev_fused = fused0;
      if (deep) {
        if (!fused0) {
          rc = enqueue_bookkeep(0, (uint32_t)cur.large, hbuf[0]);
          if (rc) return rc;
        }
        if (s1) BQS_CK(cudaEventRecord(ready[1], s));
        BQS_CK(cudaEventRecord(cev[0], s));
        last_copy.ev = cev[0];
      }
    }
    for (int level = 0;; ++level) {
      if (level > max_levels) return kErrInternal;
      const int p = level & 1, q = p ^ 1;
      P.p = p;
      const uint32_t nlarge = (uint32_t)cur.large;
      if (nlarge) {
        st.levels += 1;
        st.partition_launches += 1;
        st.active_keys += (int64_t)cur.large_keys;
      }
      const bool nets = cur.tiny || cur.small || cur.group || cur.big;
      // This level's networks: the side stream takes its dependency on the previous
      // bookkeeping (which wrote their runs) now, and the launches follow the lookahead
      // partition below, so that the host enqueues the bookkeeping, the work on the
      // critical path, first.
      const int rset = level % kSets, wset = (level + 1) % kSets;   // sets read / written
      if (nets && s1) BQS_CK(cudaStreamWaitEvent(s1, ready[rset], 0));
      auto launch_networks = [&]() -> int {
        Params Q = with_runs(P, p, rset);
        Q.p = p;
        Q.ctrl_host = nullptr;
        Q.fixed_counts = 1;
        Q.n_tiny = cur.tiny;
        Q.n_small = cur.small;
        Q.n_group = cur.group;
        Q.n_big = cur.big;
        cudaStream_t ns = s1 ? s1 : s;
        if (cur.tiny) {
          k_small_warp<KT, PAIRS><<<(int)std::min<uint32_t>((cur.tiny + 7) / 8, 16 * sms), 256, 0, ns>>>(Q, p);
          st.kernel_launches += 1;
        }
        if (cur.small || cur.group || cur.big)
          st.kernel_launches += launch_small<KT, PAIRS>(Q, p, cur.small, cur.group, cur.big, false, ns);
        st.small_segments += cur.tiny + cur.small + cur.group + cur.big;
        if (s1) {
          BQS_CK(cudaEventRecord(done[rset], s1));
          side_work[rset] = true;
        }
        BQS_CK(cudaGetLastError());
        return kOk;
      };
      if (deep) {
        // This level's bookkeeping is enqueued; next, level L+1's pivot pass, partition
        // and bookkeeping, then this level's networks, then the wait for this level's
        // counts.
        if (!nlarge) {
          if (nets) {
            rc = launch_networks();
            if (rc) return rc;
          }
          break;
        }
        P.p = q;
        if (level + 1 >= P.depth_limit || (P.pivot_rule == 1 && cur.large_keys >= 20000)) {
          k_pivot<KT, PAIRS><<<next_pivot_grid(cur), 256, 0, s>>>(P);
          st.kernel_launches += 1;
        }
        const uint64_t tiles_next = cur.large_keys / (uint64_t)tile + 4ull * nlarge + 1;
        if (fuse_ok(tiles_next, 2ull * nlarge, cur.large_keys)) {
          rc = enqueue_fused_partition(level + 1, next_part_grid(cur), 0);
          if (rc) return rc;
          prev_fused = true;
        } else {
          rc = launch_partition(q, next_part_grid(cur), 0);
          if (rc) return rc;
          rc = enqueue_bookkeep(level + 1, 2 * nlarge, hbuf[q]);
          if (rc) return rc;
          prev_fused = false;
        }
        if (s1) BQS_CK(cudaEventRecord(ready[(level + 2) % kSets], s));
        BQS_CK(cudaEventRecord(cev[q], s));
        last_copy.ev = cev[q];
        BQS_CK(cudaGetLastError());
        if (nets) {
          rc = launch_networks();
          if (rc) return rc;
        }
        BQS_CK(cudaEventSynchronize(cev[p]));
        host = hbuf[p];
        host_fresh = true;
        if (host->status) return status_code(host->status);
        cur = host->lists[q];
        if (timing) timed_work.push_back((uint32_t)cur.large != 0u);
        const unsigned long long fills = host->lists[p].fill;
        if ((uint32_t)fills) {
          Params F = P;
          F.p = p;
          F.fixed_counts = 1;
          F.n_fill = fills;
          k_fill<KT, PAIRS><<<(int)std::min<unsigned long long>(fills >> 32, 4ull * sms), 256, 0, s>>>(F, p);
          st.kernel_launches += 1;
        }
        continue;
      }
      // Bookkeeping (and single-block partitioning) write the runs of set wset, which the
      // networks of level L-2 read.
      if (nlarge || cur.local) {
        if (side_work[wset]) BQS_CK(cudaStreamWaitEvent(s, done[wset], 0));
      }
      // With the control block in host-mapped memory and no single-block partitioning
      // after it, the bookkeeping's last block copies the counts out itself.
      const bool bk_copies = nlarge && !cur.local && host_mapped;
      if (nlarge) {
        Params B = with_runs(P, q, wset);
        B.ctrl_host = bk_copies ? host : nullptr;
        k_bookkeep<KT, PAIRS><<<(int)std::min<uint32_t>((nlarge + 255) / 256, 4 * sms), 256, 0, s>>>(B);
        st.kernel_launches += 1;
      } else if (cur.local) {
        // No partition kernel cleared the next level's counts this time.
        BQS_CK(cudaMemsetAsync(&P.ctrl->lists[q], 0, sizeof(ListCounts), s));
      }
      if (cur.local) {
        st.local_segments += cur.local;
        launch_local<KT, PAIRS>(with_runs(P, q, wset), p, cur.local, s);
        st.kernel_launches += 1;
      }
      BQS_CK(cudaGetLastError());
      if (!nlarge && !cur.local) {
        if (nets) {
          rc = launch_networks();
          if (rc) return rc;
        }
        break;
      }
      if (s1) BQS_CK(cudaEventRecord(ready[wset], s));   // the runs of set wset are written
      if (!bk_copies) {
        BQS_CK(read_ctrl(P.ctrl, host, host_mapped, s));
        st.kernel_launches += 1;
      }
      BQS_CK(cudaEventRecord(counts_ev, s));
      // Lookahead: the next level's pivot pass and partition.  A segment of the next
      // level waits for the pivot pass only for a sqrt(n) sample (20000 keys and more,
      // so only if this level's large segments held that many) or at the depth limit.
      P.p = q;
      if (level + 1 >= P.depth_limit || (P.pivot_rule == 1 && cur.large_keys >= 20000)) {
        k_pivot<KT, PAIRS><<<next_pivot_grid(cur), 256, 0, s>>>(P);
        st.kernel_launches += 1;
      }
      rc = launch_partition(q, next_part_grid(cur), 0);
      if (rc) return rc;
      BQS_CK(cudaGetLastError());
      if (nets) {
        rc = launch_networks();
        if (rc) return rc;
      }
      BQS_CK(cudaEventSynchronize(counts_ev));
      host_fresh = true;
      if (host->status) return status_code(host->status);
      cur = host->lists[q];
      if (timing) timed_work.push_back((uint32_t)cur.large != 0u);
      // This level's pivot classes, now that the host knows whether there are any: the
      // launch (list length as an argument; the next partition has cleared the counts of
      // parity p, the runs stay until the bookkeeping two levels on) runs after the next
      // partition instead of before it.
      const unsigned long long fills = host->lists[p].fill;
      if ((uint32_t)fills) {
        Params F = P;
        F.p = p;
        F.fixed_counts = 1;
        F.n_fill = fills;
        k_fill<KT, PAIRS><<<(int)std::min<unsigned long long>(fills >> 32, 4ull * sms), 256, 0, s>>>(F, p);
        st.kernel_launches += 1;
      }
    }
    join();
    if (host_fresh) {
      st.moved_keys = (int64_t)host->moved_keys;
      st.equal_keys = (int64_t)host->equal_keys;
      st.small_keys = (int64_t)host->small_keys;
      st.local_keys = (int64_t)host->local_keys;
      st.fallback_pivots = (int64_t)host->fallbacks;
    } else {
      st.small_keys = (cur.tiny | cur.small | cur.group | cur.big) ? c.n : 0;
      st.local_keys = cur.local ? c.n : 0;
    }
    st.partition_bytes_per_key = (double)sizeof(U) + (PAIRS ? 4.0 : 0.0);
    if (timing && !deferred && ev_used) {
      BQS_CK(cudaEventSynchronize(evs[ev_used - 1].second));
      double ms = 0;
      for (size_t i = 0; i < ev_used && i < timed_work.size(); ++i) {
        if (!timed_work[i]) continue;
        float t = 0;
        BQS_CK(cudaEventElapsedTime(&t, evs[i].first, evs[i].second));
        ms += t;
      }
      st.partition_ms = ms;
    }
    return kOk;
  }
  // BQS_OPT_OVERLAP: each level's networks run on a second stream, beside the partition
  // levels (disjoint key ranges).  They read their list lengths from the kernel
  // arguments; `ready` marks the end of the bookkeeping that wrote their runs, `done`
  // their end, which the next bookkeeping (it rewrites those runs) and the call's
  // return wait for.
  cudaStream_t s1 = nullptr;
  cudaEvent_t ready = nullptr, done = nullptr;
  if (c.opt.overlap && counts_ev) {
    s1 = side_stream();
    ready = side_event(0);
    done = side_event(1);
    if (!s1 || !ready || !done) s1 = nullptr;
  }
  bool side_work = false;
  auto join = [&]() {
    if (side_work) cudaStreamWaitEvent(s, done, 0);
  };
  // Every way out of the call (errors included) makes the call's stream wait for the
  // networks before the scratch is returned on it.
  struct Join {
    decltype(join)& f;
    ~Join() { f(); }
  } join_on_exit{join};
  if (s1) BQS_CK(cudaEventRecord(ready, s));
  for (int level = 0;; ++level) {
    if (level > max_levels) { join(); return kErrInternal; }
    P.p = level & 1;
    const uint32_t nlarge = (uint32_t)cur.large, ntiles = (uint32_t)(cur.large >> 32);
    if (nlarge) {
      st.levels += 1;
      st.partition_launches += 1;
      st.active_keys += (int64_t)cur.large_keys;
      if (cur.todo) {
        k_pivot<KT, PAIRS><<<(int)std::min<uint32_t>(cur.todo, 8 * sms), 256, 0, s>>>(P);
        st.kernel_launches += 1;
      }
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (timing) {
        if (ev_used == evs.size()) {
          cudaEvent_t a, b;
          BQS_CK(cudaEventCreate(&a));
          BQS_CK(cudaEventCreate(&b));
          evs.emplace_back(a, b);
        }
        e0 = evs[ev_used].first; e1 = evs[ev_used].second;
        ++ev_used;
        BQS_CK(cudaEventRecord(e0, s));
      }
      P.test_stall = (level == 0 && c.opt.test_stall) ? 1 : 0;
      var.launch(P, (int)std::min<uint32_t>(ntiles, (uint32_t)part_grid_max), s, false);
      P.test_stall = 0;
      if (timing) BQS_CK(cudaEventRecord(e1, s));
      if (side_work) BQS_CK(cudaStreamWaitEvent(s, done, 0));   // the previous level's networks
    }
    if (s1 && (cur.tiny || cur.small || cur.group || cur.big)) {
      // This level's networks, beside this and the next partition level.
      BQS_CK(cudaStreamWaitEvent(s1, ready, 0));
      Params Q = P;
      Q.fixed_counts = 1;
      Q.n_tiny = cur.tiny;
      Q.n_small = cur.small;
      Q.n_group = cur.group;
      Q.n_big = cur.big;
      if (cur.tiny) {
        st.small_segments += cur.tiny;
        k_small_warp<KT, PAIRS><<<(int)std::min<uint32_t>((cur.tiny + 7) / 8, 16 * sms), 256, 0, s1>>>(Q, Q.p);
        st.kernel_launches += 1;
      }
      if (cur.small || cur.group || cur.big) {
        st.small_segments += cur.small + cur.group + cur.big;
        st.kernel_launches += launch_small<KT, PAIRS>(Q, Q.p, cur.small, cur.group, cur.big, false, s1);
      }
      BQS_CK(cudaEventRecord(done, s1));
      side_work = true;
    }
    if (nlarge) {
      k_bookkeep<KT, PAIRS><<<(int)std::min<uint32_t>((nlarge + 255) / 256, 4 * sms), 256, 0, s>>>(P);
      st.kernel_launches += 2;
    } else if (cur.local) {
      // No partition kernel clears the next level's counts this time.
      BQS_CK(cudaMemsetAsync(&P.ctrl->lists[P.p ^ 1], 0, sizeof(ListCounts), s));
    }
    if (cur.local) {   // its finished sub-segments join the next level's network lists
      st.local_segments += cur.local;
      launch_local<KT, PAIRS>(P, P.p, cur.local, s);
      st.kernel_launches += 1;
    }
    const bool more = nlarge || cur.local;
    if (s1 && more) BQS_CK(cudaEventRecord(ready, s));   // the next level's runs are written
    if (more && counts_ev) {
      // The next level's counts are final once bookkeeping and local partitioning have
      // run: read them back now, while this level's fills and sorting networks still
      // run, so the host enqueues the next level before the stream drains.
      BQS_CK(read_ctrl(P.ctrl, host, host_mapped, s));
      BQS_CK(cudaEventRecord(counts_ev, s));
    }
    if (nlarge) {
      k_fill<KT, PAIRS><<<4 * sms, 256, 0, s>>>(P, P.p);
      st.kernel_launches += 1;
    }
    if (!s1 && cur.tiny) {
      st.small_segments += cur.tiny;
      k_small_warp<KT, PAIRS><<<(int)std::min<uint32_t>((cur.tiny + 7) / 8, 16 * sms), 256, 0, s>>>(P, P.p);
      st.kernel_launches += 1;
    }
    if (!s1 && (cur.small || cur.group || cur.big)) {
      st.small_segments += cur.small + cur.group + cur.big;
      st.kernel_launches += launch_small<KT, PAIRS>(P, P.p, cur.small, cur.group, cur.big, false, s);
    }
    BQS_CK(cudaGetLastError());
    if (!more) break;
    if (counts_ev) {
      BQS_CK(cudaEventSynchronize(counts_ev));
    } else {
      BQS_CK(read_ctrl(P.ctrl, host, host_mapped, s));
      BQS_CK(cudaStreamSynchronize(s));
    }
    host_fresh = true;
    if (host->status) { join(); return status_code(host->status); }
    if (c.partition_only) {
      // split = #(< pivot); the cursor of the single segment holds it.
      unsigned long long cursor = 0;
      BQS_CK(cudaMemcpyAsync(&cursor, P.l.cursor[0], 8, cudaMemcpyDeviceToHost, s));
      BQS_CK(cudaStreamSynchronize(s));
      *c.split = (int64_t)(uint32_t)cursor;
      break;
    }
    cur = host->lists[P.p ^ 1];
  }
  join();   // the call's stream holds every kernel of the sort from here on
  if (host_fresh) {
    st.moved_keys = (int64_t)host->moved_keys;
    st.equal_keys = (int64_t)host->equal_keys;
    st.small_keys = (int64_t)host->small_keys;
    st.local_keys = (int64_t)host->local_keys;
    st.fallback_pivots = (int64_t)host->fallbacks;
  } else if (!c.partition_only) {
    // A single array that went straight to a network or the single-block partitioning:
    // nothing was read back, and the counts follow from where it was routed.
    st.small_keys = (cur.tiny | cur.small | cur.group | cur.big) ? c.n : 0;
    st.local_keys = cur.local ? c.n : 0;
  }
  st.partition_bytes_per_key = (double)sizeof(U) + (PAIRS ? 4.0 : 0.0);
  if (timing && ev_used) {
    // The partition launches are in stream order, so the last one's end event is the
    // last to complete; waiting for it (not for the whole stream) lets the call return
    // while the last level's networks still run, as an untimed call does.
    BQS_CK(cudaEventSynchronize(evs[ev_used - 1].second));
    double ms = 0;
    for (size_t i = 0; i < ev_used; ++i) {
      float t = 0;
      BQS_CK(cudaEventElapsedTime(&t, evs[i].first, evs[i].second));
      ms += t;
    }
    st.partition_ms = ms;
  }
  return kOk;
}

#undef BQS_CK

// Explicit instantiation helper used by the per-dtype translation units.
#define BQS_INSTANTIATE(KT, NAME)                                                  \
  int NAME(const Call& c, Stats& st) {                                             \
    return c.vals ? run_call<KT, true>(c, st) : run_call<KT, false>(c, st);        \
  }

}  // namespace bqs

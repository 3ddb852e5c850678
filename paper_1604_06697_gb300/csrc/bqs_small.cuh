// Small-segment sort: the GPU stand-in for the Insertionsort that finishes the paper's
// recursion (Sec. 2, "switch to Insertionsort ... when the array size is less than
// 16"): a segment of at most the small-segment cutoff is sorted by one of the register
// networks of bqs_network.cuh.  Segments of at most 256 keys: one warp each
// (k_small_warp); longer key-only segments: one warp (k_small_warps) or one small warp
// group (k_small_group) each; key-value segments: one 256-thread block each
// (k_small_block).
#pragma once

#include "bqs_kernels.cuh"

namespace bqs {

// Loads len keys of one segment (ord images, padded with the largest key) into the
// group's registers, entry e = t*R + i, through shared memory so that global reads are
// coalesced; sorts; writes the first len entries back (raw keys) the same way.
template <class KT, bool PAIRS, int R, int T>
__device__ __forceinline__ void sort_run(const Params& P, const Run& r, int t, typename KT::U* s_x,
                                         uint32_t* s_y, bool block_sync) {
  using U = typename KT::U;
  const U* src = (const U*)P.b.key[r.parity] + r.off;
  const uint32_t* vsrc = PAIRS ? P.b.val[r.parity] + r.off : nullptr;
  U* dst = (U*)P.b.final_key + r.off;
  uint32_t* vdst = PAIRS ? P.b.final_val + r.off : nullptr;
  const int len = (int)r.len;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int e = i * T + t;
    s_x[e] = e < len ? KT::ord(src[e]) : ~U(0);
    if constexpr (PAIRS) s_y[e] = e < len ? vsrc[e] : 0xFFFFFFFFu;
  }
  if (block_sync) __syncthreads(); else __syncwarp();
  U x[R];
  uint32_t y[R];
  load_row<R>(s_x + t * R, x);
  if constexpr (PAIRS) load_row<R>(s_y + t * R, y);
  if (block_sync) __syncthreads(); else __syncwarp();
  net_sort<PAIRS, R, T>(x, y, t, s_x, s_y);
  store_row<R>(s_x + t * R, x);
  if constexpr (PAIRS) store_row<R>(s_y + t * R, y);
  if (block_sync) __syncthreads(); else __syncwarp();
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int e = i * T + t;
    if (e < len) {
      dst[e] = KT::unord(s_x[e]);
      if constexpr (PAIRS) vdst[e] = s_y[e];
    }
  }
  if (block_sync) __syncthreads(); else __syncwarp();
}

// One warp per segment of at most kWarpSortMax keys (list `tiny`).
template <class KT, bool PAIRS>
__global__ void __launch_bounds__(256) k_small_warp(Params P, int p) {
  using U = typename KT::U;
  p = level_parity(P, p);
  __shared__ __align__(16) U s_x[8][kWarpSortMax];
  __shared__ __align__(16) uint32_t s_y[8][PAIRS ? kWarpSortMax : 1];
  const unsigned int count = min(P.fixed_counts ? P.n_tiny : P.ctrl->lists[p].tiny, P.l.cap_run);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (unsigned int s = blockIdx.x * 8 + warp; s < count; s += gridDim.x * 8) {
    const Run r = P.l.tiny[p][s];
    U* sx = s_x[warp];
    uint32_t* sy = PAIRS ? s_y[warp] : nullptr;
    if (r.len <= 32) sort_run<KT, PAIRS, 1, 32>(P, r, lane, sx, sy, false);
    else if (r.len <= 64) sort_run<KT, PAIRS, 2, 32>(P, r, lane, sx, sy, false);
    else if (r.len <= 128) sort_run<KT, PAIRS, 4, 32>(P, r, lane, sx, sy, false);
    else sort_run<KT, PAIRS, 8, 32>(P, r, lane, sx, sy, false);
  }
}

// ---- one warp, or one small group of warps, per small segment ---------------------------
//
// Key-only segments of the `small` list are sorted by T = 32 threads (one warp) when
// they fit 32 x R registers (R <= 32 four-byte or 16 eight-byte keys), and above that
// by one block of T = 64 (32-bit keys, R <= 32) or T = 128 (64-bit keys, R <= 16)
// threads up to kMaxSmall keys.  Compared with one
// 256-thread block and 8 keys per thread, more of the network's stages are register
// compare-exchanges (with R = 32 only index bits 5 and up need another thread), and a
// warp needs no block barrier at all.  Keys arrive striped (entry i*T + t: coalesced
// global reads) and the network holds them blocked (entry t*R + i), so they pass
// through the swizzled staging array once each way.

// Largest segment one warp sorts: 32 lanes x 32 four-byte or 16 eight-byte keys in
// registers (0: the 256-thread block kernel sorts every small segment, as for
// key-value pairs).
template <class KT, bool PAIRS>
__host__ __device__ constexpr int small_warp_max() {
  return PAIRS ? 0 : (sizeof(typename KT::U) == 4 ? 1024 : 512);
}

template <class KT>
struct SmallGroup {   // the block that sorts segments above small_warp_max()
  static constexpr int RMAX = sizeof(typename KT::U) == 4 ? 32 : 16;   // keys per thread
  static constexpr int T = kMaxSmall / RMAX;
  static constexpr int TBIG = kMaxSmallKeys / RMAX;   // the block for kMaxSmall+1 .. kMaxSmallKeys
  // Resident blocks per SM asked of the compiler.  32-bit keys: 24 warps per SM, the
  // most whose register budget (76-78 per thread) the networks fit without spilling
  // (2^28 int32 sort with cutoff 4096: 9.81 against 9.93 ms at 16 warps).  64-bit
  // keys: 16 warps (128 registers); 24 warps (72 registers) measured slower (20.53
  // against 20.15 ms at 2^28).
  static constexpr bool k32 = sizeof(typename KT::U) == 4;
  static constexpr int BLOCKS = (k32 ? 24 : 16) * 32 / T;
  static constexpr int BLOCKS_BIG = (k32 ? 24 : 16) * 32 / TBIG;
};

// Sorts len <= R*T raw keys from src (global or shared memory) into dst (the final
// buffer) with T threads; sw: their staging rows.  NB: the T threads are one of several
// groups of the block (named barriers).
// rot (flip form only): the group's warps take the network's warps rotated by rot, so
// the warp that a short segment leaves idle changes from segment to segment (and with
// it the sub-partition of the SM that waits).
template <class KT, int R, int T, bool NB = false>
__device__ __forceinline__ void group_sort_keys(const typename KT::U* src, typename KT::U* dst,
                                                int len, int t, typename KT::U* sw, int rot = 0) {
  using U = typename KT::U;
  using S = RowSwizzle<U, R>;
  auto sync = [] { sync_group<T, NB>(); };
  if constexpr (sizeof(U) == 4 && R == 32 && !NB && T > 32) {
    // The flip form of the network: only the first ceil(len / 1024) network warps hold
    // entries below len, and only they run the network (the rows of the others stay
    // padding).  Every thread still takes part in the coalesced loads and stores.
    const int act = min(T / 32, (len + 32 * R - 1) / (32 * R));
    const int tn = (t + rot * 32) & (T - 1);   // network thread index
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int e = i * T + t;
      sw[S::pos(e)] = e < len ? KT::ord(src[e]) : ~U(0);
    }
    sync();
    if ((tn >> 5) < act) {
      U x[R];
      swz_load_row<R>(sw, tn, x);
      net_sort_flip32<T>(x, tn, sw, act);
      swz_store_row<R>(sw, tn, x);
    }
    sync();
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int e = i * T + t;
      if (e < len) dst[e] = KT::unord(sw[S::pos(e)]);
    }
    sync();
    return;
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int e = i * T + t;
    sw[S::pos(e)] = e < len ? KT::ord(src[e]) : ~U(0);
  }
  sync();
  U x[R];
  uint32_t y[R];
  swz_load_row<R>(sw, t, x);
  // Exchanges between warps (T > 32) store a thread's own row before a barrier and
  // read another's after it, so the staging array doubles as their scratch.
  if constexpr (sizeof(U) == 4 && R == 32) net_sort_transposed<T, NB>(x, t, sw);
  else if constexpr (sizeof(U) == 8 && R == 16) net_sort_transposed64<T, NB>(x, t, sw);
  else net_sort_looped<R, T, U, NB>(x, t, sw);
  swz_store_row<R>(sw, t, x);
  sync();
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int e = i * T + t;
    if (e < len) dst[e] = KT::unord(sw[S::pos(e)]);
  }
  sync();
}

template <class KT, int R, int T>
__device__ __forceinline__ void group_sort_run(const Params& P, const Run& r, int t,
                                               typename KT::U* sw, int rot = 0) {
  using U = typename KT::U;
  group_sort_keys<KT, R, T>((const U*)P.b.key[r.parity] + r.off, (U*)P.b.final_key + r.off,
                            (int)r.len, t, sw, rot);
}

// Key-only small segments of kWarpSortMax+1 .. small_warp_max() keys (list `small`),
// one warp each; 5 blocks per SM for 32-bit keys (96 registers), 4 for 64-bit ones
// (the most without spilling).
template <class KT, bool PAIRS>
__global__ void __launch_bounds__(128, sizeof(typename KT::U) == 4 ? 5 : 4) k_small_warps(Params P, int p) {
  using U = typename KT::U;
  constexpr int kMax = small_warp_max<KT, PAIRS>();
  static_assert(kMax >= 512, "launched only for key-only sorts");
  p = level_parity(P, p);
  __shared__ __align__(16) U s_x[4][staging_entries<U, kMax / 32, 32>()];
  const unsigned int count = min(P.fixed_counts ? P.n_small : P.ctrl->lists[p].small, P.l.cap_run);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (unsigned int s = blockIdx.x * 4 + warp; s < count; s += gridDim.x * 4) {
    const Run r = P.l.small[p][s];
    if (r.len <= 512) group_sort_run<KT, 512 / 32, 32>(P, r, lane, s_x[warp]);
    else if constexpr (kMax >= 1024) group_sort_run<KT, 1024 / 32, 32>(P, r, lane, s_x[warp]);
  }
}

// Key-only small segments above small_warp_max() (list `group`), one group of
// SmallGroup::T threads (the whole block) each.
template <class KT, bool PAIRS>
__global__ void __launch_bounds__(SmallGroup<KT>::T, SmallGroup<KT>::BLOCKS) k_small_group(Params P, int p) {
  using U = typename KT::U;
  using G = SmallGroup<KT>;
  static_assert(!PAIRS, "launched only for key-only sorts");
  p = level_parity(P, p);
  __shared__ __align__(16) U s_x[staging_entries<U, G::RMAX, G::T>()];
  const unsigned int count = min(P.fixed_counts ? P.n_group : P.ctrl->lists[p].group, P.l.cap_run);
  for (unsigned int s = blockIdx.x; s < count; s += gridDim.x) {
    const Run r = P.l.group[p][s];
    if (r.len * 2 <= kMaxSmall) group_sort_run<KT, G::RMAX / 2, G::T>(P, r, threadIdx.x, s_x);
    else group_sort_run<KT, G::RMAX, G::T>(P, r, threadIdx.x, s_x);
  }
}

// Key-only small segments of kMaxSmall+1 .. kMaxSmallKeys keys (list `big`, small
// cutoffs above kMaxSmall), one block of SmallGroup::TBIG threads each: the same network
// with twice the threads, one more phase of exchanges between warps.
template <class KT, bool PAIRS>
__global__ void __launch_bounds__(SmallGroup<KT>::TBIG, SmallGroup<KT>::BLOCKS_BIG) k_small_big(Params P, int p) {
  using U = typename KT::U;
  using G = SmallGroup<KT>;
  static_assert(!PAIRS, "launched only for key-only sorts");
  p = level_parity(P, p);
  __shared__ __align__(16) U s_x[staging_entries<U, G::RMAX, G::TBIG>()];
  const unsigned int count = min(P.fixed_counts ? P.n_big : P.ctrl->lists[p].big, P.l.cap_run);
  for (unsigned int s = blockIdx.x, k = 0; s < count; s += gridDim.x, ++k)
    group_sort_run<KT, G::RMAX, G::TBIG>(P, P.l.big[p][s], threadIdx.x, s_x, (int)((blockIdx.x + k) & 3));
}

// ---- key-value segments as packed 64-bit keys ------------------------------------------
//
// (key, payload) pairs are ordered lexicographically.  When the order images of a
// segment's keys span less than 2^32 (always for 32-bit keys), the pair maps to
// ((ord(key) - min) << 32) | payload, a 64-bit integer in the same order, and the
// segment is sorted by the key-only 64-bit networks; other segments are left to the
// 256-thread key-value network (k_small_block), which makes the same test.

// Smallest ord image of segment r's keys and whether the pairs pack (block-wide; every
// thread of the block must call it; s_red holds 2 * (blockDim.x / 32) entries).
template <class KT>
__device__ __forceinline__ bool pairs_pack(const Params& P, const Run& r, typename KT::U& kmin,
                                           typename KT::U* s_red) {
  using U = typename KT::U;
  if constexpr (sizeof(U) == 4) {
    kmin = 0;
    return true;
  } else {
    const U* src = (const U*)P.b.key[r.parity] + r.off;
    U lo = ~U(0), hi = 0;
    for (int i = threadIdx.x; i < (int)r.len; i += blockDim.x) {
      const U k = KT::ord(src[i]);
      lo = k < lo ? k : lo;
      hi = k > hi ? k : hi;
    }
    for (int o = 16; o; o >>= 1) {
      const U a = (U)__shfl_xor_sync(~0u, (unsigned long long)lo, o);
      const U b = (U)__shfl_xor_sync(~0u, (unsigned long long)hi, o);
      lo = a < lo ? a : lo;
      hi = b > hi ? b : hi;
    }
    const int warps = blockDim.x >> 5, w = threadIdx.x >> 5;
    __syncthreads();                                  // s_red free from earlier use
    if ((threadIdx.x & 31) == 0) { s_red[w] = lo; s_red[warps + w] = hi; }
    __syncthreads();
    lo = s_red[0];
    hi = s_red[warps];
    for (int i = 1; i < warps; ++i) {
      lo = s_red[i] < lo ? s_red[i] : lo;
      hi = s_red[warps + i] > hi ? s_red[warps + i] : hi;
    }
    kmin = lo;
    return hi - lo <= (U)0xFFFFFFFFull;
  }
}

template <class KT, int R, int T>
__device__ __forceinline__ void packed_pairs_run(const Params& P, const Run& r, typename KT::U kmin,
                                                 uint64_t* sw) {
  using U = typename KT::U;
  using S = RowSwizzle<uint64_t, R>;
  const int t = threadIdx.x;
  const U* src = (const U*)P.b.key[r.parity] + r.off;
  const uint32_t* vsrc = P.b.val[r.parity] + r.off;
  U* dst = (U*)P.b.final_key + r.off;
  uint32_t* vdst = P.b.final_val + r.off;
  const int len = (int)r.len;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int e = i * T + t;
    sw[S::pos(e)] = e < len ? ((uint64_t)(KT::ord(src[e]) - kmin) << 32) | vsrc[e] : ~0ull;
  }
  __syncthreads();
  uint64_t x[R];
  swz_load_row<R>(sw, t, x);
  if constexpr (R == 16) net_sort_transposed64<T>(x, t, sw);
  else net_sort_looped<R, T>(x, t, sw);
  swz_store_row<R>(sw, t, x);
  __syncthreads();
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int e = i * T + t;
    if (e < len) {
      const uint64_t v = sw[S::pos(e)];
      dst[e] = KT::unord(kmin + (U)(v >> 32));
      vdst[e] = (uint32_t)v;
    }
  }
  __syncthreads();
}

// Key-value segments of the `small` list whose keys pack, one 128-thread block each.
template <class KT>
__global__ void __launch_bounds__(128, 4) k_small_pairs_packed(Params P, int p) {
  using U = typename KT::U;
  constexpr int T = 128;
  p = level_parity(P, p);
  __shared__ __align__(16) uint64_t s_w[staging_entries<uint64_t, kMaxSmall / T, T>()];
  __shared__ U s_red[2 * (T / 32)];
  const unsigned int count = min(P.fixed_counts ? P.n_small : P.ctrl->lists[p].small, P.l.cap_run);
  for (unsigned int s = blockIdx.x; s < count; s += gridDim.x) {
    const Run r = P.l.small[p][s];
    U kmin;
    if (!pairs_pack<KT>(P, r, kmin, s_red)) continue;   // k_small_block's
    if (r.len <= 512) packed_pairs_run<KT, 4, T>(P, r, kmin, s_w);
    else if (r.len <= 1024) packed_pairs_run<KT, 8, T>(P, r, kmin, s_w);
    else packed_pairs_run<KT, 16, T>(P, r, kmin, s_w);
  }
}

// One 256-thread block per segment of kWarpSortMax+1 .. kMaxSmall keys (list `small`):
// key-value sorts (with small_sort = 0 only the segments whose keys do not pack), and
// key-only sorts with BQS_OPT_SMALL_SORT = 1.
template <class KT, bool PAIRS>
__global__ void __launch_bounds__(256) k_small_block(Params P, int p) {
  using U = typename KT::U;
  p = level_parity(P, p);
  __shared__ __align__(16) U s_x[kMaxSmall];
  __shared__ __align__(16) uint32_t s_y[PAIRS ? kMaxSmall : 1];
  __shared__ U s_red[PAIRS ? 16 : 1];
  const unsigned int count = min(P.fixed_counts ? P.n_small : P.ctrl->lists[p].small, P.l.cap_run);
  for (unsigned int s = blockIdx.x; s < count; s += gridDim.x) {
    const Run r = P.l.small[p][s];
    if constexpr (PAIRS) {
      U kmin;
      if (P.small_sort == 0 && pairs_pack<KT>(P, r, kmin, s_red)) continue;   // packed
    }
    if (r.len <= 512) sort_run<KT, PAIRS, 2, 256>(P, r, threadIdx.x, s_x, s_y, true);
    else if (r.len <= 1024) sort_run<KT, PAIRS, 4, 256>(P, r, threadIdx.x, s_x, s_y, true);
    else sort_run<KT, PAIRS, 8, 256>(P, r, threadIdx.x, s_x, s_y, true);
  }
}

}  // namespace bqs

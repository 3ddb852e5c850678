// Small-segment sort: a bitonic sorting network (Batcher 1968) held in registers.
//
// This is the GPU stand-in for the Insertionsort that finishes the paper's recursion
// (Sec. 2, "switch to Insertionsort ... when the array size is less than 16"): a
// segment of at most the small-segment cutoff is loaded into shared memory, padded
// with the largest order key to m = 2^k entries, and sorted by a fixed network with no
// data-dependent branches.  Each thread holds R consecutive entries in registers
// (entry e = thread * R + i), so
//   * exchanges between entries less than R apart are register compare-exchanges,
//   * exchanges between threads of one warp use __shfl_xor_sync,
//   * only exchanges between warps go through shared memory.
// Segments of at most 256 keys are sorted by one warp each (k_small_warp); longer ones
// by one 256-thread block each (k_small_block).
#pragma once

#include "bqs_kernels.cuh"

namespace bqs {

template <class U>
__device__ __forceinline__ U shfl_xor_any(U x, int d) {
  if constexpr (sizeof(U) == 8) {
    return (U)__shfl_xor_sync(~0u, (unsigned long long)x, d);
  } else {
    return (U)__shfl_xor_sync(~0u, (unsigned)x, d);
  }
}

// A thread's row of R consecutive entries in shared memory, moved with 16-byte (or
// 8-byte) accesses: a warp then touches consecutive 16-byte words and no bank twice
// beyond the minimum number of wavefronts.
template <int R, class U>
__device__ __forceinline__ void store_row(U* dst, const U (&x)[R]) {
  constexpr int BYTES = R * (int)sizeof(U);
  if constexpr (BYTES % 16 == 0) {
    constexpr int PER = 16 / (int)sizeof(U);
#pragma unroll
    for (int c = 0; c < BYTES / 16; ++c) {
      union { uint4 v; U e[PER]; } u;
#pragma unroll
      for (int e = 0; e < PER; ++e) u.e[e] = x[c * PER + e];
      reinterpret_cast<uint4*>(dst)[c] = u.v;
    }
  } else if constexpr (BYTES == 8) {
    union { uint2 v; U e[8 / sizeof(U)]; } u;
#pragma unroll
    for (int e = 0; e < R; ++e) u.e[e] = x[e];
    *reinterpret_cast<uint2*>(dst) = u.v;
  } else {
#pragma unroll
    for (int e = 0; e < R; ++e) dst[e] = x[e];
  }
}

template <int R, class U>
__device__ __forceinline__ void load_row(const U* src, U (&x)[R]) {
  constexpr int BYTES = R * (int)sizeof(U);
  if constexpr (BYTES % 16 == 0) {
    constexpr int PER = 16 / (int)sizeof(U);
#pragma unroll
    for (int c = 0; c < BYTES / 16; ++c) {
      union { uint4 v; U e[PER]; } u;
      u.v = reinterpret_cast<const uint4*>(src)[c];
#pragma unroll
      for (int e = 0; e < PER; ++e) x[c * PER + e] = u.e[e];
    }
  } else if constexpr (BYTES == 8) {
    union { uint2 v; U e[8 / sizeof(U)]; } u;
    u.v = *reinterpret_cast<const uint2*>(src);
#pragma unroll
    for (int e = 0; e < R; ++e) x[e] = u.e[e];
  } else {
#pragma unroll
    for (int e = 0; e < R; ++e) x[e] = src[e];
  }
}

template <class U>
__device__ __forceinline__ U umin_(U a, U b) { return a < b ? a : b; }
template <class U>
__device__ __forceinline__ U umax_(U a, U b) { return a < b ? b : a; }

// Ascending compare-exchange of two register entries: afterwards a <= b.
template <bool PAIRS, class U>
__device__ __forceinline__ void cx_up(U& a, uint32_t& va, U& b, uint32_t& vb) {
  if constexpr (PAIRS) {
    const bool sw = elem_less<PAIRS>(b, vb, a, va);
    const U ta = sw ? b : a, tb = sw ? a : b;
    const uint32_t tva = sw ? vb : va, tvb = sw ? va : vb;
    a = ta; b = tb; va = tva; vb = tvb;
  } else {
    const U lo = umin_(a, b), hi = umax_(a, b);
    a = lo;
    b = hi;
  }
}

// Keeps the smaller (keep_min) or larger of an entry and its partner's.
template <bool PAIRS, class U>
__device__ __forceinline__ void keep_one(U& x, uint32_t& y, U p, uint32_t pv, bool keep_min) {
  if constexpr (PAIRS) {
    const bool take = elem_less<PAIRS>(p, pv, x, y) == keep_min;
    x = take ? p : x;
    y = take ? pv : y;
  } else {
    x = keep_min ? umin_(x, p) : umax_(x, p);
  }
}

// Sorts the m = R*T entries held as x[R], y[R] by T participating threads (t = thread
// index within the group), ascending.  Entries are ord images (+ payloads), so bitwise
// complement reverses their order: during merge phase k every entry whose index has
// bit k set is kept complemented, which turns the descending half-merges of Batcher's
// network into ascending ones and leaves every compare-exchange a plain min/max.
// s_x / s_y: shared scratch of m entries, used only for exchanges between warps.
template <bool PAIRS, int R, int T, class U>
__device__ __forceinline__ void net_sort(U (&x)[R], uint32_t (&y)[R], int t, U* s_x, uint32_t* s_y) {
  constexpr int M = R * T;
#pragma unroll
  for (int k = 2; k <= M; k <<= 1) {
    // Entering phase k: flip the entries whose complement state changes.
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int e = t * R + i;
      const bool before = (k >= 4) && ((e & (k >> 1)) != 0);
      const bool now = (k < M) && ((e & k) != 0);
      const U m = (before != now) ? ~U(0) : U(0);
      x[i] ^= m;
      if constexpr (PAIRS) y[i] ^= (uint32_t)m;
    }
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j < R) {
        // Both entries of every pair are in this thread.
#pragma unroll
        for (int i = 0; i < R; ++i)
          if ((i & j) == 0) cx_up<PAIRS>(x[i], y[i], x[i | j], y[i | j]);
      } else if (j < 32 * R) {
        // Partner entry: same register of lane t ^ (j / R); the lower index keeps the min.
        const int d = j / R;
        const bool keep_min = (t & d) == 0;
#pragma unroll
        for (int i = 0; i < R; ++i) {
          const U p = shfl_xor_any(x[i], d);
          const uint32_t pv = PAIRS ? __shfl_xor_sync(~0u, y[i], d) : 0u;
          keep_one<PAIRS>(x[i], y[i], p, pv, keep_min);
        }
      } else {
        // Partner in another warp: exchange rows through shared memory.
        const int d = j / R;
        const bool keep_min = (t & d) == 0;
        store_row<R>(s_x + t * R, x);
        if constexpr (PAIRS) store_row<R>(s_y + t * R, y);
        __syncthreads();
        U p[R];
        uint32_t pv[R];
        load_row<R>(s_x + (t ^ d) * R, p);
        if constexpr (PAIRS) load_row<R>(s_y + (t ^ d) * R, pv);
#pragma unroll
        for (int i = 0; i < R; ++i) keep_one<PAIRS>(x[i], y[i], p[i], PAIRS ? pv[i] : 0u, keep_min);
        __syncthreads();
      }
    }
  }
}

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
  const unsigned int count = min(P.ctrl->lists[p].tiny, P.l.cap_run);
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

// One 256-thread block per segment of kWarpSortMax+1 .. kMaxSmall keys (list `small`).
template <class KT, bool PAIRS>
__global__ void __launch_bounds__(256) k_small_block(Params P, int p) {
  using U = typename KT::U;
  p = level_parity(P, p);
  __shared__ __align__(16) U s_x[kMaxSmall];
  __shared__ __align__(16) uint32_t s_y[PAIRS ? kMaxSmall : 1];
  const unsigned int count = min(P.ctrl->lists[p].small, P.l.cap_run);
  for (unsigned int s = blockIdx.x; s < count; s += gridDim.x) {
    const Run r = P.l.small[p][s];
    if (r.len <= 512) sort_run<KT, PAIRS, 2, 256>(P, r, threadIdx.x, s_x, s_y, true);
    else if (r.len <= 1024) sort_run<KT, PAIRS, 4, 256>(P, r, threadIdx.x, s_x, s_y, true);
    else sort_run<KT, PAIRS, 8, 256>(P, r, threadIdx.x, s_x, s_y, true);
  }
}

}  // namespace bqs

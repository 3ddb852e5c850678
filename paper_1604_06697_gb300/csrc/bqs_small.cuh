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

// Compare-exchange of two register entries: afterwards (a, b) is ordered ascending
// when `up`, descending otherwise.
template <bool PAIRS, class U>
__device__ __forceinline__ void cx(U& a, uint32_t& va, U& b, uint32_t& vb, bool up) {
  const bool sw = up ? elem_less<PAIRS>(b, vb, a, va) : elem_less<PAIRS>(a, va, b, vb);
  const U ta = sw ? b : a, tb = sw ? a : b;
  a = ta;
  b = tb;
  if constexpr (PAIRS) {
    const uint32_t tva = sw ? vb : va, tvb = sw ? va : vb;
    va = tva;
    vb = tvb;
  }
}

// Sorts the m = R*T entries held as x[R], y[R] by the T = blockDim-participating threads
// (t = thread index within the group).  s_x / s_y: shared scratch of m entries, used
// only for exchanges between warps (T > 32).  Entries are ord images (+ payloads).
template <bool PAIRS, int R, int T, class U>
__device__ __forceinline__ void net_sort(U (&x)[R], uint32_t (&y)[R], int t, U* s_x, uint32_t* s_y) {
  constexpr int M = R * T;
#pragma unroll
  for (int k = 2; k <= M; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j < R) {
        // Both entries of every pair are in this thread.
#pragma unroll
        for (int i = 0; i < R; ++i) {
          if ((i & j) == 0) {
            const bool up = (k < R) ? ((i & k) == 0) : (((t * R) & k) == 0);
            cx<PAIRS>(x[i], y[i], x[i | j], y[i | j], up);
          }
        }
      } else if (j < 32 * R) {
        // Partner entry: same register of lane t ^ (j / R).
        const int d = j / R;
        const bool keep_min = (((t & d) == 0) == (((t * R) & k) == 0));
#pragma unroll
        for (int i = 0; i < R; ++i) {
          const U p = shfl_xor_any(x[i], d);
          const uint32_t pv = PAIRS ? __shfl_xor_sync(~0u, y[i], d) : 0u;
          const bool take = elem_less<PAIRS>(p, pv, x[i], y[i]) == keep_min;
          x[i] = take ? p : x[i];
          if constexpr (PAIRS) y[i] = take ? pv : y[i];
        }
      } else {
        // Partner in another warp: exchange through shared memory.
        const int d = j / R;
        const bool keep_min = (((t & d) == 0) == (((t * R) & k) == 0));
#pragma unroll
        for (int i = 0; i < R; ++i) {
          s_x[t * R + i] = x[i];
          if constexpr (PAIRS) s_y[t * R + i] = y[i];
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < R; ++i) {
          const U p = s_x[(t ^ d) * R + i];
          const uint32_t pv = PAIRS ? s_y[(t ^ d) * R + i] : 0u;
          const bool take = elem_less<PAIRS>(p, pv, x[i], y[i]) == keep_min;
          x[i] = take ? p : x[i];
          if constexpr (PAIRS) y[i] = take ? pv : y[i];
        }
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
  constexpr int M = R * T;
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
#pragma unroll
  for (int i = 0; i < R; ++i) {
    x[i] = s_x[t * R + i];
    y[i] = PAIRS ? s_y[t * R + i] : 0u;
  }
  if (block_sync) __syncthreads(); else __syncwarp();
  net_sort<PAIRS, R, T>(x, y, t, s_x, s_y);
#pragma unroll
  for (int i = 0; i < R; ++i) {
    s_x[t * R + i] = x[i];
    if constexpr (PAIRS) s_y[t * R + i] = y[i];
  }
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

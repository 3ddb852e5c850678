// sm_103a kernels of the level-synchronous BlockQuicksort.
//
//   k_init_*      first work lists from the caller's array / segments
//   k_pivot       pivots that need a whole block (sqrt(n) sample, depth fallback)
//   (the partition step itself, Algorithm 3 per tile, is k_partition_tma in bqs_tma.cuh)
//   k_bookkeep    children of every partitioned segment (Quicksort main loop)
//   k_fill        writes the class equal to a pivot into the final buffer
// The small-segment sorting network is in bqs_small.cuh.
#pragma once

#include "bqs_common.cuh"
#include "bqs_network.cuh"

namespace bqs {

// ---- small helpers --------------------------------------------------------------------

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__host__ __device__ __forceinline__ int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

__device__ __forceinline__ int64_t isqrt64(int64_t n) {
  int64_t r = (int64_t)sqrt((double)n);
  while (r * r > n) --r;
  while ((r + 1) * (r + 1) <= n) ++r;
  return r;
}

// ---- pivot selection ---------------------------------------------------------------------

template <class KT, bool PAIRS>
struct Elem {
  typename KT::U k;  // ord image
  uint32_t v;
};

template <class KT, bool PAIRS>
__device__ __forceinline__ Elem<KT, PAIRS> load_elem(const typename KT::U* keys,
                                                     const uint32_t* vals, int64_t i) {
  Elem<KT, PAIRS> e;
  e.k = KT::ord(keys[i]);
  e.v = PAIRS ? vals[i] : 0u;
  return e;
}

template <class KT, bool PAIRS>
__device__ __forceinline__ bool lt(const Elem<KT, PAIRS>& a, const Elem<KT, PAIRS>& b) {
  return elem_less<PAIRS>(a.k, a.v, b.k, b.v);
}

// Median of three values (Sec. 2): the middle one of the ordered triple.
template <class KT, bool PAIRS>
__device__ __forceinline__ Elem<KT, PAIRS> median3(Elem<KT, PAIRS> a, Elem<KT, PAIRS> b, Elem<KT, PAIRS> c) {
  if (lt(b, a)) { auto t = a; a = b; b = t; }
  if (lt(c, b)) { auto t = b; b = c; c = t; }
  if (lt(b, a)) { auto t = a; a = b; b = t; }
  return b;
}

// Ascending compare-exchange of two sample entries.
template <class KT, bool PAIRS>
__device__ __forceinline__ void cx_elem(Elem<KT, PAIRS>& a, Elem<KT, PAIRS>& b) {
  if (lt(b, a)) { const auto t = a; a = b; b = t; }
}

// Median of five values: the middle entry after a fixed 9-comparator sorting network
// for five inputs (Knuth, TAOCP vol. 3, Sec. 5.3.4), so every index is a constant and
// the five values stay in registers.
template <class KT, bool PAIRS>
__device__ __forceinline__ Elem<KT, PAIRS> median5(Elem<KT, PAIRS> (&e)[5]) {
  cx_elem(e[0], e[1]); cx_elem(e[3], e[4]); cx_elem(e[2], e[4]);
  cx_elem(e[2], e[3]); cx_elem(e[1], e[4]); cx_elem(e[0], e[3]);
  cx_elem(e[0], e[2]); cx_elem(e[1], e[3]); cx_elem(e[1], e[2]);
  return e[2];
}

// The pivot rules of Sec. 4 ("Different Pivot Selection Methods"), BQS_OPT_PIVOT:
//   0 median-of-3 of (first, middle, last)     4 median-of-3-medians-of-3
//   1 median-of-sqrt(n) (see below)            5 median-of-3-medians-of-5
//   2 median-of-5                              6 median-of-5-medians-of-5
//   3 median-of-23
// Samples other than rule 0's are k equally spaced keys, key i at
// b + floor((2i+1) len / (2k)); a median of medians takes k = G*K of them in G groups
// of K consecutive sample keys.  Every rule uses median-of-3 below 64 keys.  The
// sqrt(n) rule takes median-of-5-medians-of-5 below 20000 keys and above that the
// median of floor(sqrt(len))|1 spaced keys, sampled by k_pivot.

// Median of K (odd) spaced keys: the middle of the sorted sample.
template <class KT, bool PAIRS, int K>
__device__ Elem<KT, PAIRS> median_spaced(const typename KT::U* keys, const uint32_t* vals,
                                         int64_t b, int64_t len) {
  Elem<KT, PAIRS> e[K];
  for (int i = 0; i < K; ++i)
    e[i] = load_elem<KT, PAIRS>(keys, vals, b + ((2 * (int64_t)i + 1) * len) / (2 * K));
  for (int i = 1; i < K; ++i) {        // insertion sort of the sample
    Elem<KT, PAIRS> x = e[i];
    int j = i;
    while (j > 0 && lt(x, e[j - 1])) { e[j] = e[j - 1]; --j; }
    e[j] = x;
  }
  return e[K / 2];
}

// Median of G medians of K consecutive sample keys (G, K in {3, 5}).
template <class KT, bool PAIRS, int G, int K>
__device__ Elem<KT, PAIRS> median_of_medians(const typename KT::U* keys, const uint32_t* vals,
                                             int64_t b, int64_t len) {
  Elem<KT, PAIRS> m[G];
#pragma unroll
  for (int g = 0; g < G; ++g) {
    Elem<KT, PAIRS> e[K];
#pragma unroll
    for (int j = 0; j < K; ++j)
      e[j] = load_elem<KT, PAIRS>(keys, vals, b + ((2 * (int64_t)(K * g + j) + 1) * len) / (2 * G * K));
    if constexpr (K == 3) m[g] = median3<KT, PAIRS>(e[0], e[1], e[2]);
    else m[g] = median5<KT, PAIRS>(e);
  }
  if constexpr (G == 3) return median3<KT, PAIRS>(m[0], m[1], m[2]);
  else return median5<KT, PAIRS>(m);
}

// A pivot one thread evaluates: every rule below 20000 keys, all but sqrt(n) above.
template <class KT, bool PAIRS>
__device__ Elem<KT, PAIRS> rule_pivot(const typename KT::U* keys, const uint32_t* vals, int64_t b,
                                      int64_t len, int rule) {
  if (rule == 0 || len < 64)
    return median3<KT, PAIRS>(load_elem<KT, PAIRS>(keys, vals, b),
                              load_elem<KT, PAIRS>(keys, vals, b + len / 2),
                              load_elem<KT, PAIRS>(keys, vals, b + len - 1));
  switch (rule) {
    case 2: return median_spaced<KT, PAIRS, 5>(keys, vals, b, len);
    case 3: return median_spaced<KT, PAIRS, 23>(keys, vals, b, len);
    case 4: return median_of_medians<KT, PAIRS, 3, 3>(keys, vals, b, len);
    case 5: return median_of_medians<KT, PAIRS, 3, 5>(keys, vals, b, len);
    default: return median_of_medians<KT, PAIRS, 5, 5>(keys, vals, b, len);   // 1 and 6
  }
}

// Returns false when the segment needs k_pivot instead (a sqrt(n) sample, or the
// depth-limit fallback).
template <class KT, bool PAIRS>
__device__ bool inline_pivot(const Params& P, int64_t b, int64_t len, int parity, int depth,
                             uint64_t& pkey, uint32_t& pval) {
  if (depth >= P.depth_limit) return false;
  if (P.pivot_rule == 1 && len >= 20000) return false;
  const Elem<KT, PAIRS> piv = rule_pivot<KT, PAIRS>((const typename KT::U*)P.b.key[parity],
                                                    P.b.val[parity], b, len, P.pivot_rule);
  pkey = (uint64_t)KT::unord(piv.k);
  pval = piv.v;
  return true;
}

// Warp-cooperative append of up to two child segments per lane (`act[c]` children with
// len > 0) to the lists of level q: the sorting network (len <= small_cutoff), the
// single-block partitioning (len <= local_cutoff) or another partition level.  Every
// lane of the warp must call it.  The warp reserves its slots with one atomic per list
// for both children at once, and the atomics of all lists are in flight together
// (lanes 0..5 take the five run lists and `todo`, lane 31 the packed large-segment
// atomic, so a large segment's slot and first tile come from one 64-bit atomic and
// tile0 grows with the slot index).  A large segment's pivot is chosen here, while
// the atomics are in flight, when one thread can do it; otherwise the segment is
// queued on `todo` for k_pivot.
template <class KT, bool PAIRS>
__device__ void route_pair(const Params& P, int q, const bool act[2], const int64_t off[2],
                           const int64_t len[2], int parity, int depth, bool count_keys = true) {
  Ctrl* c = P.ctrl;
  ListCounts& lc = c->lists[q];
  const int lane = threadIdx.x & 31;
  const unsigned below = lanemask_lt();
  int kind[2];            // 0 tiny, 1 small, 2 local, 3 group, 4 big, 5 large, -1 none
  bool needs_kernel[2];   // large, with its pivot left to k_pivot
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const bool has = act[h] && len[h] > 0;
    const bool sorted_now = has && len[h] <= P.small_cutoff;
    const bool tiny = sorted_now && len[h] <= kWarpSortMax;        // one warp per segment
    const bool big = sorted_now && len[h] > kMaxSmall;             // one larger warp group (key-only)
    const bool group = sorted_now && !big && len[h] > P.group_min; // one warp group per segment
    const bool local = has && !sorted_now && len[h] <= P.local_cutoff;
    kind[h] = !has ? -1 : tiny ? 0 : big ? 4 : group ? 3 : sorted_now ? 1 : local ? 2 : 5;
    needs_kernel[h] = kind[h] == 5 &&
                      (depth >= P.depth_limit || (P.pivot_rule == 1 && len[h] >= 20000));
  }

  // Per-list masks and counts (uniform over the warp), then the reservations.
  unsigned m0[5], m1[5], cnt[6];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    m0[k] = __ballot_sync(~0u, kind[0] == k);
    m1[k] = __ballot_sync(~0u, kind[1] == k);
    cnt[k] = __popc(m0[k]) + __popc(m1[k]);
  }
  const unsigned t0 = __ballot_sync(~0u, needs_kernel[0]), t1 = __ballot_sync(~0u, needs_kernel[1]);
  cnt[5] = __popc(t0) + __popc(t1);
  // (With net_acc the four network sizes share one list and one counter.)
  unsigned int* const netc = P.net_acc ? &P.net_acc->small : nullptr;
  unsigned int* ctr = lane == 0 ? (netc ? netc : &lc.tiny) : lane == 1 ? (netc ? netc : &lc.small)
                    : lane == 2 ? &lc.local : lane == 3 ? (netc ? netc : &lc.group)
                    : lane == 4 ? (netc ? netc : &lc.big) : &lc.todo;
  unsigned want = 0;
#pragma unroll
  for (int k = 0; k < 6; ++k) want = lane == k ? cnt[k] : want;
  unsigned int rb = 0;
  if (lane < 6 && want) rb = atomicAdd(ctr, want);

  unsigned long long own[2], lkeys = 0;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const bool large = kind[h] == 5;
    const unsigned long long tiles = large ? (unsigned long long)tile_count(off[h], len[h], P.tile) : 0ull;
    own[h] = large ? (1ull | (tiles << 32)) : 0ull;
    lkeys += large ? (unsigned long long)len[h] : 0ull;
  }
  unsigned long long v = own[0] + own[1];
  const bool any_large = __any_sync(~0u, v != 0ull);
  unsigned long long lbase = 0;
  if (any_large) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {          // inclusive scan of the packed (count, tiles)
      const unsigned long long x = __shfl_up_sync(~0u, v, o);
      if (lane >= o) v += x;
      lkeys += __shfl_xor_sync(~0u, lkeys, o);
    }
    if (lane == 31) {
      lbase = atomicAdd(&lc.large, v);
      atomicAdd(&lc.large_keys, lkeys);
    }
  }
  if (count_keys) {
    unsigned sk = 0, lk = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const unsigned l = kind[h] >= 0 && kind[h] <= 4 ? (unsigned)len[h] : 0u;
      sk += kind[h] == 2 ? 0u : l;
      lk += kind[h] == 2 ? l : 0u;
    }
    sk = __reduce_add_sync(~0u, sk);   // <= 64 * 2^14
    lk = __reduce_add_sync(~0u, lk);
    if (lane == 0 && sk) atomicAdd(&c->small_keys, (unsigned long long)sk);
    if (lane == 1 && lk) atomicAdd(&c->local_keys, (unsigned long long)lk);
  }

  // Pivots of the large children while the reservations are in flight.
  uint64_t pkey[2] = {0, 0};
  uint32_t pval[2] = {0, 0};
#pragma unroll
  for (int h = 0; h < 2; ++h)
    if (kind[h] == 5 && !needs_kernel[h]) {
      const Elem<KT, PAIRS> piv = rule_pivot<KT, PAIRS>((const typename KT::U*)P.b.key[parity],
                                                        P.b.val[parity], off[h], len[h], P.pivot_rule);
      pkey[h] = (uint64_t)KT::unord(piv.k);
      pval[h] = piv.v;
    }

#pragma unroll
  for (int k = 0; k < 5; ++k) {
    if (!cnt[k]) continue;
    const unsigned int base = __shfl_sync(~0u, rb, k);
    Run* list = k == 0 ? P.l.tiny[q] : k == 1 ? P.l.small[q] : k == 2 ? P.l.local[q]
              : k == 3 ? P.l.group[q] : P.l.big[q];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (kind[h] != k) continue;
      const unsigned int slot = base + (h ? __popc(m0[k]) + __popc(m1[k] & below) : __popc(m0[k] & below));
      if (slot < P.l.cap_run) {
        Run r;
        r.off = off[h]; r.len = len[h]; r.parity = parity; r.pad = depth;   // depth: local runs
        list[slot] = r;
      } else {
        atomicExch(&c->status, kStatusOverflow);
      }
    }
  }

  if (!any_large) return;
  lbase = __shfl_sync(~0u, lbase, 31);
  const unsigned int tb = __shfl_sync(~0u, rb, 5);
  unsigned long long at = lbase + v - own[0] - own[1];   // exclusive prefix within the warp
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const unsigned int slot = (unsigned int)at;
    if (kind[h] == 5) {
      const bool fits = slot < P.l.cap_large;
      if (fits) {
        Seg sg;
        sg.off = off[h]; sg.len = len[h]; sg.pkey = pkey[h]; sg.pval = pval[h];
        sg.depth = depth; sg.parity = parity;
        sg.tile0 = (unsigned int)(at >> 32);
        P.l.large[q][slot] = sg;
        P.l.cursor[q][slot] = 0ull;
        P.l.tdone[q][slot] = 0ull;
      } else {
        atomicExch(&c->status, kStatusOverflow);
      }
      if (needs_kernel[h]) {
        // An overflowed segment (the call fails anyway) points k_pivot at slot 0, which
        // the overflow implies was reserved and written.
        const unsigned int ts = tb + (h ? __popc(t0) + __popc(t1 & below) : __popc(t0 & below));
        if (ts < P.l.cap_large) P.l.todo[q][ts] = fits ? slot : 0u;
      }
    }
    at += own[h];
  }
}

// One child segment per lane: route_pair with the second child absent.
template <class KT, bool PAIRS>
__device__ __forceinline__ void route_warp(const Params& P, int q, bool active, int64_t off,
                                           int64_t len, int parity, int depth, bool count_keys = true) {
  const bool act[2] = {active, false};
  const int64_t o[2] = {off, 0};
  const int64_t l[2] = {len, 0};
  route_pair<KT, PAIRS>(P, q, act, o, l, parity, depth, count_keys);
}

// ---- first work lists --------------------------------------------------------------------

template <class KT, bool PAIRS>
__global__ void k_init_single(Params P, int64_t n) {
  if (blockIdx.x == 0 && threadIdx.x < 32) route_warp<KT, PAIRS>(P, 0, threadIdx.x == 0, 0, n, 0, 0);
}

// A single segment with a caller-given pivot (bqs_partition): always partitioned.
template <class KT>
__global__ void k_init_partition(Params P, int64_t n, uint64_t pkey) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Seg s;
    s.off = 0; s.len = n; s.pkey = pkey; s.pval = 0; s.depth = 0; s.parity = 0; s.tile0 = 0;
    P.l.large[0][0] = s;
    P.l.cursor[0][0] = 0ull;
    P.l.tdone[0][0] = 0ull;
    P.ctrl->lists[0].large = 1ull | ((unsigned long long)((n - 1) / P.tile + 1) << 32);
    P.ctrl->lists[0].large_keys = (unsigned long long)n;
  }
}

// One thread per caller segment: check the offsets, then route the segment.
template <class KT, bool PAIRS>
__global__ void __launch_bounds__(256) k_init_segments(Params P, const int64_t* __restrict__ offs,
                                                       int64_t nseg) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nseg; base += stride) {
    const int64_t i = base + threadIdx.x;
    bool ok = false;
    int64_t a = 0, b = 0;
    if (i < nseg) {
      a = offs[i];
      b = offs[i + 1];
      ok = a >= 0 && b >= a;
      if (!ok) atomicExch(&P.ctrl->status, kStatusInvalid);
    }
    route_warp<KT, PAIRS>(P, 0, ok, a, b - a, 0, 0);
  }
}

// ---- pivot selection kernel ---------------------------------------------------------------

// Pivots that need more than one thread (the list `todo`):
//  * sqrt rule (Sec. 4) at 20000 keys and more: the median of k = floor(sqrt(len))|1
//    equally spaced keys (k capped at kMaxSample); samples of up to 256 keys are
//    sorted in registers by one warp each, larger ones by the whole block (two
//    entries per thread in registers, stages between warps through shared memory);
//  * a segment at the depth limit gets the midpoint of its ord-key range (payload
//    range when all its keys are equal): each such level halves the range, so the
//    recursion depth stays bounded by the key width (the role Heapsort plays in Sec. 2).
// All other pivots are chosen by route_warp when the segment is created.
// Shared memory of the pivot pass (one 256-thread block).
template <class KT, bool PAIRS>
struct PivotSmem {
  static constexpr int kBlockList = 64;
  alignas(16) typename KT::U k[512];            // staging rows of the sample sort
  alignas(16) uint32_t v[PAIRS ? 512 : 1];
  typename KT::U red[2][8];
  uint32_t redv[2][8];
  unsigned int blk[kBlockList];                 // segments this block's warps leave to it
  int nblk;
};

// The pivot pass over the `todo` list of parity pp, by every 256-thread block of the
// grid (k_pivot, and one step of the cooperative sort).
template <class KT, bool PAIRS>
__device__ void pivot_pass(const Params& P, int pp, PivotSmem<KT, PAIRS>& sm) {
  using U = typename KT::U;
  using E = Elem<KT, PAIRS>;
  static_assert(kMaxSample < 512, "two sample entries per thread of 256");
  U* s_k = sm.k;
  uint32_t* s_v = sm.v;
  auto& s_red = sm.red;
  auto& s_redv = sm.redv;
  constexpr int kBlockList = PivotSmem<KT, PAIRS>::kBlockList;
  unsigned int* s_blk = sm.blk;
  int& s_nblk = sm.nblk;

  const unsigned int count = min(P.ctrl->lists[pp].todo, P.l.cap_large);
  Seg* segs = P.l.large[pp];
  auto sample_size = [](int64_t len) {
    const int64_t k = isqrt64(len) | 1;
    return k > kMaxSample ? (int64_t)kMaxSample : k;
  };

  // Samples of up to 256 keys: one warp per segment sorts them in registers (8 per
  // lane, a bitonic network without block barriers) and reads off the median.  The
  // other segments a warp meets go on the block's list for the block phase below.
  // Block b's warps take the entries b, b + gridDim, b + 2 gridDim, ..., so the
  // segments left to the blocks spread over all of them.
  if (threadIdx.x == 0) s_nblk = 0;
  __syncthreads();
  const unsigned int nw = blockDim.x >> 5;
  {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (unsigned int i = blockIdx.x + warp * gridDim.x; i < count; i += gridDim.x * nw) {
      const unsigned int s = P.l.todo[pp][i];
      const Seg sg = segs[s];
      const int64_t k = sample_size(sg.len);
      if (sg.depth >= P.depth_limit || k > 256) {
        if (lane == 0) {
          const int j = atomicAdd(&s_nblk, 1);
          if (j < kBlockList) s_blk[j] = s;
        }
        continue;
      }
      const U* keys = (const U*)P.b.key[sg.parity];
      const uint32_t* vals = P.b.val[sg.parity];
      U x[8];
      uint32_t y[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int e = lane * 8 + r;
        if (e < k) {
          const int64_t pos = sg.off + ((2 * (int64_t)e + 1) * sg.len) / (2 * k);
          x[r] = KT::ord(keys[pos]);
          y[r] = PAIRS ? vals[pos] : 0u;
        } else {
          x[r] = ~U(0);
          y[r] = 0xFFFFFFFFu;
        }
      }
      net_sort<PAIRS, 8, 32>(x, y, lane, (U*)nullptr, (uint32_t*)nullptr);
      const int med = (int)((k - 1) / 2);
      U mk = x[0];
      uint32_t mv = y[0];
#pragma unroll
      for (int r = 1; r < 8; ++r)
        if (r == (med & 7)) { mk = x[r]; mv = y[r]; }
      if constexpr (sizeof(U) == 8) mk = (U)__shfl_sync(~0u, (unsigned long long)mk, med >> 3);
      else mk = (U)__shfl_sync(~0u, (unsigned)mk, med >> 3);
      mv = __shfl_sync(~0u, mv, med >> 3);
      if (lane == 0) {
        segs[s].pkey = (uint64_t)KT::unord(mk);
        segs[s].pval = PAIRS ? mv : 0u;
      }
    }
  }

  // Larger samples and the depth-limit fallback: the whole block per segment, for the
  // segments its warps listed, or, when the list overflowed, for every such segment
  // among the entries its warps visited (the same set, read again).
  __syncthreads();
  const int nblk = s_nblk;
  const bool listed = nblk <= kBlockList;
  const unsigned int rounds = listed ? (unsigned int)nblk : (count + gridDim.x - 1) / gridDim.x;
  for (unsigned int r = 0; r < rounds; ++r) {
    unsigned int s;
    if (listed) {
      s = s_blk[r];
    } else {
      const unsigned int i = blockIdx.x + r * gridDim.x;
      if (i >= count) continue;
      s = P.l.todo[pp][i];
    }
    const Seg sg = segs[s];
    if (sg.depth < P.depth_limit && sample_size(sg.len) <= 256) continue;   // done above
    const U* keys = (const U*)P.b.key[sg.parity];
    const uint32_t* vals = P.b.val[sg.parity];
    const int64_t b = sg.off, len = sg.len;
    E piv;
    if (sg.depth >= P.depth_limit) {
      // Midpoint of the ord-key range (then of the payload range when it is empty).
      U kmin = ~U(0), kmax = 0;
      for (int64_t i = threadIdx.x; i < len; i += blockDim.x) {
        U k = KT::ord(keys[b + i]);
        kmin = k < kmin ? k : kmin;
        kmax = k > kmax ? k : kmax;
      }
      for (int o = 16; o; o >>= 1) {
        U a = __shfl_xor_sync(~0u, kmin, o), c = __shfl_xor_sync(~0u, kmax, o);
        kmin = a < kmin ? a : kmin;
        kmax = c > kmax ? c : kmax;
      }
      if ((threadIdx.x & 31) == 0) { s_red[0][threadIdx.x >> 5] = kmin; s_red[1][threadIdx.x >> 5] = kmax; }
      __syncthreads();
      kmin = s_red[0][0]; kmax = s_red[1][0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        kmin = s_red[0][w] < kmin ? s_red[0][w] : kmin;
        kmax = s_red[1][w] > kmax ? s_red[1][w] : kmax;
      }
      piv.k = kmin + (kmax - kmin) / 2;
      piv.v = 0xFFFFFFFFu;  // keys == midpoint join the left side
      if (PAIRS && kmin == kmax) {
        uint32_t vmin = 0xFFFFFFFFu, vmax = 0;
        for (int64_t i = threadIdx.x; i < len; i += blockDim.x) {
          uint32_t v = vals[b + i];
          vmin = min(vmin, v);
          vmax = max(vmax, v);
        }
        for (int o = 16; o; o >>= 1) {
          vmin = min(vmin, __shfl_xor_sync(~0u, vmin, o));
          vmax = max(vmax, __shfl_xor_sync(~0u, vmax, o));
        }
        __syncthreads();
        if ((threadIdx.x & 31) == 0) { s_redv[0][threadIdx.x >> 5] = vmin; s_redv[1][threadIdx.x >> 5] = vmax; }
        __syncthreads();
        vmin = s_redv[0][0]; vmax = s_redv[1][0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
          vmin = min(vmin, s_redv[0][w]);
          vmax = max(vmax, s_redv[1][w]);
        }
        piv.v = vmin + (vmax - vmin) / 2;
      }
      if (threadIdx.x == 0) atomicAdd(&P.ctrl->fallbacks, 1ull);
      if (threadIdx.x == 0) {
        segs[s].pkey = (uint64_t)KT::unord(piv.k);
        segs[s].pval = piv.v;
      }
    } else {
      // 257 .. kMaxSample samples: 512 entries, two per thread in registers, sorted by
      // the block's bitonic network (stages between warps through s_k / s_v).
      const int64_t k = sample_size(len);
      U x[2];
      uint32_t y[2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int e = (int)threadIdx.x * 2 + i;
        if (e < k) {
          const int64_t pos = b + ((2 * (int64_t)e + 1) * len) / (2 * k);
          x[i] = KT::ord(keys[pos]);
          y[i] = PAIRS ? vals[pos] : 0u;
        } else {
          x[i] = ~U(0);
          y[i] = 0xFFFFFFFFu;
        }
      }
      net_sort<PAIRS, 2, 256>(x, y, (int)threadIdx.x, s_k, s_v);
      const int med = (int)((k - 1) / 2);
      if ((int)threadIdx.x == med / 2) {
        segs[s].pkey = (uint64_t)KT::unord(x[med & 1]);
        segs[s].pval = PAIRS ? y[med & 1] : 0u;
      }
    }
    __syncthreads();
  }
}

template <class KT, bool PAIRS>
__global__ void __launch_bounds__(256) k_pivot(Params P) {
  __shared__ PivotSmem<KT, PAIRS> sm;
  pivot_pass<KT, PAIRS>(P, level_parity(P, P.p), sm);
}

// ---- children of the partitioned segments ------------------------------------------------

// The bookkeeping of one partitioned segment per lane (`active` lanes; every lane of
// the warp calls it), given the segment and its final counts: statistics, the pivot
// class (written here when short, else queued for k_fill), and both children routed
// to the lists of level q.
template <class KT, bool PAIRS>
__device__ void bookkeep_children(const Params& P, int p, int q, bool active, const Seg& sg,
                                  int64_t nlt, int64_t ngt) {
  const int lane = threadIdx.x & 31;
  const int64_t neq = active ? sg.len - nlt - ngt : 0;
  if (!active) { nlt = 0; ngt = 0; }
  // Statistics, one atomic per warp.
  unsigned long long moved = (unsigned long long)(nlt + ngt), eq = (unsigned long long)neq;
  for (int o = 16; o; o >>= 1) {
    moved += __shfl_xor_sync(~0u, moved, o);
    eq += __shfl_xor_sync(~0u, eq, o);
  }
  if (lane == 0) {
    atomicAdd(&P.ctrl->moved_keys, moved);
    atomicAdd(&P.ctrl->equal_keys, eq);
  }
  // The keys equal to the pivot are final.  A short run is written here; longer runs
  // are queued for k_fill (packed atomic).
  if (active && neq > 0 && neq <= kInlineFill) {
    using U = typename KT::U;
    U* fk = (U*)P.b.final_key + sg.off + nlt;
    for (int64_t j = 0; j < neq; ++j) {
      fk[j] = (U)sg.pkey;
      if constexpr (PAIRS) P.b.final_val[sg.off + nlt + j] = sg.pval;
    }
  }
  const bool fills = active && neq > kInlineFill;
  if (__any_sync(~0u, fills)) {
    const unsigned long long ftiles = fills ? (unsigned long long)((neq + kFillTile - 1) / kFillTile) : 0ull;
    unsigned long long v = fills ? (1ull | (ftiles << 32)) : 0ull;
    const unsigned long long own = v;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long x = __shfl_up_sync(~0u, v, o);
      if (lane >= o) v += x;
    }
    unsigned long long fb = 0;
    if (lane == 31) fb = atomicAdd(P.net_acc ? &P.net_acc->fill : &P.ctrl->lists[p].fill, v);
    fb = __shfl_sync(~0u, fb, 31);
    if (fills) {
      const unsigned long long old = fb + v - own;
      const unsigned int slot = (unsigned int)old;
      if (slot < P.l.cap_fill) {
        Fill f;
        f.off = sg.off + nlt; f.len = neq; f.pkey = sg.pkey; f.pval = sg.pval;
        f.tile0 = (unsigned int)(old >> 32);
        P.l.fill[p][slot] = f;
      } else {
        atomicExch(&P.ctrl->status, kStatusOverflow);
      }
    }
  }
  if (P.route_children) {   // both sides exclude the pivot class (Sec. 2)
    const bool act[2] = {active, active};
    const int64_t off[2] = {sg.off, sg.off + sg.len - ngt};
    const int64_t len[2] = {nlt, ngt};
    route_pair<KT, PAIRS>(P, q, act, off, len, sg.parity ^ 1, sg.depth + 1);
  }
}

// bookkeep_children for the segment in slot s of the level's list, with the counts
// the partition tiles accumulated in its cursor.
template <class KT, bool PAIRS>
__device__ void bookkeep_warp(const Params& P, int p, int q, bool active, unsigned int s) {
  Seg sg{};
  int64_t nlt = 0, ngt = 0;
  if (active) {
    sg = P.l.large[p][s];
    const unsigned long long cur = P.l.cursor[p][s];
    nlt = (uint32_t)cur;
    ngt = (uint32_t)(cur >> 32);
  }
  bookkeep_children<KT, PAIRS>(P, p, q, active, sg, nlt, ngt);
}

// Fused bookkeeping (partition kernel, small levels): each finished tile adds
// (#< | #> << 24 | 1 << 48) of its keys to its segment's word in `tdone`, with one
// acquire-release atomic; the tile that brings the tile count to the segment's total
// has the segment's final counts in hand.  The host fuses only levels of fewer than
// 2^24 keys, so the fields cannot overflow.
constexpr int kDoneShift = 24;
__host__ __device__ constexpr unsigned long long done_word(uint32_t nlt, uint32_t ngt) {
  return (unsigned long long)nlt | ((unsigned long long)ngt << kDoneShift) |
         (1ull << (2 * kDoneShift));
}
constexpr unsigned long long kFusedMaxKeys = 1ull << kDoneShift;

__device__ __forceinline__ unsigned int atomic_add_acq_rel_u32(unsigned int* a, unsigned int v) {
  unsigned int old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(a), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ unsigned long long atomic_add_acq_rel(unsigned long long* a,
                                                                 unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(a), "l"(v) : "memory");
  return old;
}

// Copies the control block (the next level's counts, this level's fills, the
// statistics) to host-mapped memory; every thread of the block calls it.  With
// clear_p >= 0 the counts of lists[clear_p] (the level's consumed lists) are cleared
// after the copy, for the next level's bookkeeping.
__device__ __forceinline__ void copy_ctrl_out(const Params& P, int clear_p) {
  __threadfence();
  static_assert(sizeof(Ctrl) % 8 == 0, "control block in 8-byte words");
  const volatile unsigned long long* src = reinterpret_cast<const volatile unsigned long long*>(P.ctrl);
  unsigned long long* dst = reinterpret_cast<unsigned long long*>(P.ctrl_host);
  // No system-scope fence: the host reads the block only after an event behind this
  // kernel has completed, which orders the kernel's writes before it.
  for (int i = threadIdx.x; i < (int)(sizeof(Ctrl) / 8); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    P.ctrl->bk_done = 0;
    if (clear_p >= 0) clear_counts(&P.ctrl->lists[clear_p]);
  }
}

template <class KT, bool PAIRS>
__global__ void __launch_bounds__(256) k_bookkeep(Params P) {
  const int p = level_parity(P, P.p), q = p ^ 1;
  const unsigned int count = min((unsigned int)P.ctrl->lists[p].large, P.l.cap_large);
  const unsigned int stride = gridDim.x * blockDim.x;
  for (unsigned int base = blockIdx.x * blockDim.x; base < count; base += stride)
    bookkeep_warp<KT, PAIRS>(P, p, q, base + threadIdx.x < count, base + threadIdx.x);
  if (P.ctrl_host) {
    // The last block to finish copies the control block out (a single block is last).
    __shared__ bool s_last;
    if (gridDim.x > 1) {
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&P.ctrl->bk_done, 1u) == gridDim.x - 1;
      }
      __syncthreads();
      if (!s_last) return;
    } else {
      __syncthreads();
    }
    copy_ctrl_out(P, -1);
  }
}

// ---- keys equal to a pivot ----------------------------------------------------------------

template <class KT, bool PAIRS>
__global__ void __launch_bounds__(256) k_fill(Params P, int p) {
  using U = typename KT::U;
  __shared__ uint32_t s_f;
  p = level_parity(P, p);
  const unsigned long long lc = P.fixed_counts ? P.n_fill : P.ctrl->lists[p].fill;
  const uint32_t count = min((uint32_t)lc, P.l.cap_fill), tiles = (uint32_t)(lc >> 32);
  const Fill* fills = P.l.fill[p];
  if (count == 0) return;
  U* fk = (U*)P.b.final_key;
  for (uint32_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    if (threadIdx.x == 0) {
      uint32_t lo = 0, hi = count;
      while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (fills[mid].tile0 <= t) lo = mid; else hi = mid;
      }
      s_f = lo;
    }
    __syncthreads();
    const Fill f = fills[s_f];
    const int64_t b = f.off + (int64_t)(t - f.tile0) * kFillTile;
    const int64_t e = min(b + kFillTile, f.off + f.len);
    for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
      fk[i] = (U)f.pkey;
      if constexpr (PAIRS) P.b.final_val[i] = f.pval;
    }
    __syncthreads();
  }
}

}  // namespace bqs

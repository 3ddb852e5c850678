// Single-launch sort of a small array: the whole level loop inside one cooperative
// kernel.
//
// For arrays of up to a few million keys the host-driven level loop costs more than the
// work: every level is a handful of launches and a read-back of the next level's
// counts, while the keys (a few MB) sit in L2.  Here one persistent grid (every block
// resident, cudaLaunchCooperativeKernel) runs every level of the same recursion
// (Sec. 2, Algorithm 1, breadth first; the block partition step of Sec. 3 per tile)
// and meets at one grid-wide barrier per level instead of returning to the host:
//
//   level L (large segments of parity p, the next level's of parity q = p ^ 1):
//     [pivot samples of the segments queued for one, when there are any; barrier]
//     partition every tile of the large segments; the block that completes a
//     segment's last tile does its bookkeeping at once: large children go to the
//     lists of q, network runs and pivot-class fills to lists kept for the end of
//     the launch;                                                         barrier
//   after the last level: every network run and every fill.
//
// Tiles, network runs and fill ranges touch disjoint key ranges, and a small segment's
// keys stay where its level left them, so the networks can wait for the end.  Every
// barrier wait is bounded: when one gives up, the block records BQS_ERR_TIMEOUT in the
// status word and returns (the kernel has no asynchronous copies to wait for), so a
// failure never hangs the device.
#pragma once

#include "bqs_small.cuh"
#include "bqs_tma.cuh"

namespace bqs {

constexpr int kCoopThreads = 256;

template <class KT>
struct CoopShape {
  using U = typename KT::U;
  using G = SmallGroup<KT>;
  static constexpr int KPT = sizeof(U) == 4 ? 16 : 8;      // keys per thread of a tile
  static constexpr int TILE = kCoopThreads * KPT;
  static constexpr int WARPS = kCoopThreads / 32;
  static constexpr int kWarpStage = staging_entries<U, small_warp_max<KT, false>() / 32, 32>();
  static constexpr int cmax(int a, int b) { return a > b ? a : b; }
  // One shared-memory area serves, phase by phase, as the tile's staging, the warps'
  // network rows or the warp groups' network rows.
  static constexpr int kEntries =
      cmax(cmax(TILE, WARPS * kWarpSortMax),
           cmax(WARPS * kWarpStage,
                cmax((kCoopThreads / G::T) * staging_entries<U, G::RMAX, G::T>(),
                     (kCoopThreads / G::TBIG) * staging_entries<U, G::RMAX, G::TBIG>())));
  static constexpr size_t smem = (size_t)kEntries * sizeof(U);
  static_assert(smem <= 48 * 1024, "static launch without a shared-memory attribute");
};

// Bounded barrier of all blocks of a cooperative launch, on two words of the control
// block (cleared by the host before the launch).  The last block to arrive resets the
// count and advances the generation the others wait on.
// With clear_p >= 0 the last block to arrive also empties the counts of lists[clear_p]
// before it releases the others.
__device__ __forceinline__ bool coop_grid_sync(Ctrl* c, uint32_t limit, int* s_ok, int clear_p = -1) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = &c->bar_gen;
    const unsigned int g = *gen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(&c->bar_count, 1u) + 1u == gridDim.x) {
      if (clear_p >= 0) clear_counts(&c->lists[clear_p]);
      atomicExch(&c->bar_count, 0u);
      __threadfence();
      atomicAdd(&c->bar_gen, 1u);
    } else {
      for (uint32_t it = 0; *gen == g; ++it) {
        if (it >= limit) {
          atomicExch(&c->status, kStatusTimeout);
          ok = 0;
          break;
        }
        if (it > 64) __nanosleep(64);
      }
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// The block partition step (Sec. 3) on tile t of the level's tile space: the same
// computation as the TMA-fed kernel (outcome counts in registers, warp scan, one packed
// atomic per tile, staging in output order, coalesced write-out), with the keys read
// straight from global memory (L2-resident at these sizes), and the fused bookkeeping
// of the partition kernel's small-level instantiation.
template <class KT>
__device__ __forceinline__ void coop_tile(const Params& P, int p, uint32_t t, uint32_t nseg,
                                          typename KT::U* s_out, uint32_t* s_wcnt,
                                          unsigned long long* s_base, uint32_t* s_idx,
                                          unsigned long long* s_word) {
  using U = typename KT::U;
  using CT = typename Cmp<KT>::T;
  using CS = CoopShape<KT>;
  constexpr int KPT = CS::KPT, TILE = CS::TILE, WARPS = CS::WARPS, T = kCoopThreads;
  constexpr int VEC = 16 / (int)sizeof(U), NV = KPT / VEC;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const Seg* segs = P.l.large[p];
  if (warp == 0) {
    // The segment that owns tile t (the last one whose first tile is at most t): a
    // 32-way search, one round of 32 parallel probes per factor of 32 in nseg.
    uint32_t lo = 0, hi = nseg;
    while (hi - lo > 1) {
      const uint32_t step = (hi - lo + 31) / 32;
      const uint32_t idx = lo + lane * step;
      const unsigned m = __ballot_sync(~0u, idx < hi && segs[idx].tile0 <= t);
      const uint32_t k = 31 - __clz(m);   // lane 0 always qualifies: segs[lo].tile0 <= t
      lo += k * step;
      hi = min(hi, lo + step);
    }
    if (lane == 0) *s_idx = lo;
  }
  __syncthreads();
  const uint32_t si = *s_idx;
  const Seg sg = segs[si];
  const int64_t abase = tile_origin(sg.off) + (int64_t)(t - sg.tile0) * TILE;
  const int lo = (int)(max(abase, sg.off) - abase);
  const int hi = (int)(min(abase + TILE, sg.off + sg.len) - abase);
  const U* src = (const U*)P.b.key[sg.parity] + abase;
  const CT cp = Cmp<KT>::of((U)sg.pkey);

  // Scan phase: keys outside the segment count as equal to the pivot.
  U key[KPT];
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    const int i0 = (j * T + tid) * VEC;
    if (i0 >= lo && i0 + VEC <= hi) {
      union { uint4 v; U e[VEC]; } u;
      u.v = *reinterpret_cast<const uint4*>(src + i0);
#pragma unroll
      for (int e = 0; e < VEC; ++e) key[j * VEC + e] = u.e[e];
    } else {
#pragma unroll
      for (int e = 0; e < VEC; ++e)
        key[j * VEC + e] = (i0 + e >= lo && i0 + e < hi) ? src[i0 + e] : (U)sg.pkey;
    }
  }
  CT kc[KPT];
  uint32_t cl = 0, cg = 0;
#pragma unroll
  for (int r = 0; r < KPT; ++r) {
    kc[r] = Cmp<KT>::of(key[r]);
    cl += kc[r] < cp;
    cg += cp < kc[r];
  }
  const uint32_t own = cl | (cg << 16);
  uint32_t incl = own;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(~0u, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_wcnt[warp] = incl;
  __syncthreads();
  uint32_t off_lt = 0, off_gt = 0, nlt = 0, ngt = 0;
#pragma unroll
  for (int w = 0; w < WARPS; ++w) {
    const uint32_t c = s_wcnt[w];
    if (w < warp) { off_lt += c & 0xFFFF; off_gt += c >> 16; }
    nlt += c & 0xFFFF;
    ngt += c >> 16;
  }
  unsigned long long my_base = 0;
  if (tid == 0)
    my_base = atomicAdd(&P.l.cursor[p][si], (unsigned long long)nlt | ((unsigned long long)ngt << 32));
  // Rearrangement into output order in shared memory, then to the other buffer.
  const uint32_t excl = incl - own;
  uint32_t pl = off_lt + (excl & 0xFFFF), pg = nlt + off_gt + (excl >> 16);
#pragma unroll
  for (int r = 0; r < KPT; ++r) {
    const bool l = kc[r] < cp, g = cp < kc[r];
    if (l) s_out[pl] = key[r];
    if (g) s_out[pg] = key[r];
    pl += l;
    pg += g;
  }
  if (tid == 0) *s_base = my_base;
  __syncthreads();
  const unsigned long long base = *s_base;
  U* dst = (U*)P.b.key[sg.parity ^ 1];
  U* dl = dst + sg.off + (int64_t)(uint32_t)base;
  U* dr = dst + sg.off + sg.len - (int64_t)(uint32_t)(base >> 32) - ngt;
  for (uint32_t j = tid; j < nlt; j += T) dl[j] = s_out[j];
  for (uint32_t j = tid; j < ngt; j += T) dr[j] = s_out[nlt + j];
  // Completion: the tile's write-out is published (block barrier, then thread 0's
  // acquire-release atomic on the segment's completion word, see done_word); the tile
  // that completes the segment's count does its bookkeeping with warp 0, from the
  // segment's descriptor and the word's totals.
  __syncthreads();
  if (tid == 0) {
    const unsigned long long mine = done_word(nlt, ngt);
    const unsigned long long tot = atomic_add_acq_rel(&P.l.tdone[p][si], mine) + mine;
    *s_word = (uint32_t)(tot >> (2 * kDoneShift)) == (uint32_t)tile_count(sg.off, sg.len, TILE) ? tot : 0ull;
  }
  __syncthreads();
  const unsigned long long tot = *s_word;
  if (tot && warp == 0) {
    constexpr unsigned long long kField = (1ull << kDoneShift) - 1;
    bookkeep_children<KT, false>(P, p, p ^ 1, lane == 0, sg, (int64_t)(tot & kField),
                                 (int64_t)((tot >> kDoneShift) & kField));
  }
  // The next tile's first barrier (after its segment search) orders the reuse of s_out,
  // s_wcnt, s_base, s_idx and s_word.
}

// The network runs of every level, one list of `count` runs of all sizes, sorted by the
// block's warps (runs of at most small_warp_max() keys, one warp each) and warp groups
// (longer ones; named barriers per group, or the block barrier when a group is the
// whole block), one size class per pass.  Block b takes every gridDim-th run of a pass.
template <class KT>
__device__ __forceinline__ void coop_networks(const Params& P, uint32_t count,
                                              typename KT::U* stage) {
  using U = typename KT::U;
  using G = SmallGroup<KT>;
  using CS = CoopShape<KT>;
  constexpr int T = kCoopThreads, W = CS::WARPS;
  constexpr int kMax = small_warp_max<KT, false>();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const Run* runs = P.l.small[0];
  for (uint32_t s = blockIdx.x * W + warp; s < count; s += gridDim.x * W) {
    const Run r = runs[s];
    if (r.len > kWarpSortMax) continue;
    U* sx = stage + warp * kWarpSortMax;
    if (r.len <= 32) sort_run<KT, false, 1, 32>(P, r, lane, sx, nullptr, false);
    else if (r.len <= 64) sort_run<KT, false, 2, 32>(P, r, lane, sx, nullptr, false);
    else if (r.len <= 128) sort_run<KT, false, 4, 32>(P, r, lane, sx, nullptr, false);
    else sort_run<KT, false, 8, 32>(P, r, lane, sx, nullptr, false);
  }
  __syncthreads();
  for (uint32_t s = blockIdx.x * W + warp; s < count; s += gridDim.x * W) {
    const Run r = runs[s];
    if (r.len <= kWarpSortMax || r.len > P.group_min) continue;
    U* sw = stage + warp * CS::kWarpStage;
    if (r.len <= 512) group_sort_run<KT, 512 / 32, 32>(P, r, lane, sw);
    else if constexpr (kMax >= 1024) group_sort_run<KT, 1024 / 32, 32>(P, r, lane, sw);
  }
  __syncthreads();
  {
    constexpr int NG = T / G::T;
    const int g = tid / G::T, gt = tid % G::T;
    U* sw = stage + g * staging_entries<U, G::RMAX, G::T>();
    for (uint32_t s = blockIdx.x * NG + g; s < count; s += gridDim.x * NG) {
      const Run r = runs[s];
      if (r.len <= P.group_min || r.len > kMaxSmall) continue;
      const U* src = (const U*)P.b.key[r.parity] + r.off;
      U* dst = (U*)P.b.final_key + r.off;
      if (r.len * 2 <= kMaxSmall)
        group_sort_keys<KT, G::RMAX / 2, G::T, (G::T < T)>(src, dst, (int)r.len, gt, sw);
      else
        group_sort_keys<KT, G::RMAX, G::T, (G::T < T)>(src, dst, (int)r.len, gt, sw);
    }
  }
  __syncthreads();
  {
    constexpr int NG = T / G::TBIG;
    const int g = tid / G::TBIG, gt = tid % G::TBIG;
    U* sw = stage + g * staging_entries<U, G::RMAX, G::TBIG>();
    for (uint32_t s = blockIdx.x * NG + g; s < count; s += gridDim.x * NG) {
      const Run r = runs[s];
      if (r.len <= kMaxSmall) continue;
      group_sort_keys<KT, G::RMAX, G::TBIG, (G::TBIG < T)>((const U*)P.b.key[r.parity] + r.off,
                                                          (U*)P.b.final_key + r.off, (int)r.len, gt, sw);
    }
  }
  __syncthreads();
}

// The pivot classes of the fill list of parity p: every key of each range is its
// segment's pivot (equal keys are bit-identical under the total order).
template <class KT>
__device__ __forceinline__ void coop_fills(const Params& P, int p, unsigned long long fill_count,
                                           uint32_t* s_idx) {
  using U = typename KT::U;
  const uint32_t count = min((uint32_t)fill_count, P.l.cap_fill), tiles = (uint32_t)(fill_count >> 32);
  const Fill* fills = P.l.fill[p];
  U* fk = (U*)P.b.final_key;
  for (uint32_t t = blockIdx.x; t < tiles && count; t += gridDim.x) {
    if (threadIdx.x == 0) {
      uint32_t lo = 0, hi = count;
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (fills[mid].tile0 <= t) lo = mid; else hi = mid;
      }
      *s_idx = lo;
    }
    __syncthreads();
    const Fill f = fills[*s_idx];
    const int64_t b = f.off + (int64_t)(t - f.tile0) * kFillTile;
    const int64_t e = min(b + kFillTile, f.off + f.len);
    for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) fk[i] = (U)f.pkey;
    __syncthreads();
  }
}

// The cooperative sort of keys[0, n) (key-only).  Launched with every block resident;
// the host has cleared the control block and pointed the network-run and fill lists
// of both parities at the lists kept for the end (P.net_acc).
template <class KT>
__global__ void __launch_bounds__(kCoopThreads, 2) k_coop_sort(Params P, int64_t n, int max_levels) {
  using U = typename KT::U;
  extern __shared__ __align__(16) unsigned char coop_smem[];
  U* stage = reinterpret_cast<U*>(coop_smem);
  __shared__ PivotSmem<KT, false> psm;
  __shared__ uint32_t s_wcnt[CoopShape<KT>::WARPS];
  __shared__ unsigned long long s_base, s_word;
  __shared__ uint32_t s_idx;
  __shared__ int s_ok;
  Ctrl* c = P.ctrl;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;

  if (blockIdx.x == 0 && threadIdx.x < 32) route_warp<KT, false>(P, 0, threadIdx.x == 0, 0, n, 0, 0);
  // Failure-path test (BQS_OPT_TEST_STALL): block 0 never arrives at the first barrier,
  // so every other block's bounded wait runs out.
  if (P.test_stall && blockIdx.x == 0) return;
  if (!coop_grid_sync(c, P.wait_limit, &s_ok)) return;
  int level = 0;
  for (;; ++level) {
    const int p = level & 1;
    // Every block reads the same counts: nothing writes lists[p] between the last
    // barrier and the end of this level's tiles (the bookkeeping appends to lists[q]).
    const volatile ListCounts* vl = &c->lists[p];
    const unsigned long long large = vl->large, large_keys = vl->large_keys;
    const uint32_t todo = vl->todo;
    const uint32_t nlarge = min((uint32_t)large, P.l.cap_large);
    const uint32_t ntiles = nlarge ? (uint32_t)(large >> 32) : 0u;
    if (*(volatile int*)&c->status != 0) break;
    if (!nlarge) break;
    if (level > max_levels) {
      if (lead) atomicExch(&c->status, kStatusOverflow);
      break;
    }
    if (todo) {   // sample pivots (sqrt(n) rule) and depth-limit fallbacks
      pivot_pass<KT, false>(P, p, psm);
      if (!coop_grid_sync(c, P.wait_limit, &s_ok)) return;
    }
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x)
      coop_tile<KT>(P, p, t, nlarge, stage, s_wcnt, &s_base, &s_idx, &s_word);
    if (lead) {
      c->levels_run += 1;
      c->active_total += large_keys;
    }
    // The last block to arrive empties lists[p]: the next level's bookkeeping appends
    // to them.
    if (!coop_grid_sync(c, P.wait_limit, &s_ok, p)) return;
  }
  // Every level's network runs and pivot-class fills.
  const volatile ListCounts* acc = P.net_acc;
  const uint32_t nruns = min(acc->small, P.l.cap_run);
  const unsigned long long fills = acc->fill;
  coop_networks<KT>(P, nruns, stage);
  coop_fills<KT>(P, 0, fills, &s_idx);
  if (lead) {
    c->level = level;
    c->small_runs = nruns;
  }
}

}  // namespace bqs

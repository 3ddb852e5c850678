// Single-launch sort of a small array: the whole level loop inside one cooperative
// kernel.
//
// For arrays of up to a few million keys the host-driven level loop costs more than the
// work: every level is a handful of launches and a read-back of the next level's
// counts, while the keys (a few MB) sit in L2.  Here one persistent grid (every block
// resident, cudaLaunchCooperativeKernel) runs every level of the same recursion
// (Sec. 2, Algorithm 1, breadth first; the block partition step of Sec. 3 per tile)
// and meets at a grid-wide barrier instead of returning to the host:
//
//   level L (lists of parity p, the next level's of parity q = p ^ 1):
//     [pivot samples of the segments queued for one, when there are any; barrier]
//     partition every tile of the large segments, sort the small segments that level
//     L-1 produced, write the pivot classes that level L-1 found;       barrier
//     bookkeeping: the children of every partitioned segment go to the lists of q,
//     pivot classes to q's fill list;                                    barrier
//
// Tiles, small segments and fill ranges of one level touch disjoint key ranges, so the
// first phase needs no order among them.  Every barrier wait is bounded: when one gives
// up, the block records BQS_ERR_TIMEOUT in the status word and returns (the kernel has
// no asynchronous copies to wait for), so a failure never hangs the device.
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
__device__ __forceinline__ bool coop_grid_sync(Ctrl* c, uint32_t limit, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = &c->bar_gen;
    const unsigned int g = *gen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(&c->bar_count, 1u) + 1u == gridDim.x) {
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
// straight from global memory (L2-resident at these sizes).
template <class KT>
__device__ __forceinline__ void coop_tile(const Params& P, int p, uint32_t t, uint32_t nseg,
                                          typename KT::U* s_out, uint32_t* s_wcnt,
                                          unsigned long long* s_base, uint32_t* s_idx) {
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
  // The next tile's first barrier (after its segment search) orders the reuse of s_out,
  // s_wcnt, s_base and s_idx; the caller adds one after its last tile.
}

// The small segments of the lists of parity p, sorted by the block's warps (segments of
// at most small_warp_max() keys, one warp each) and warp groups (longer ones; named
// barriers per group, or the block barrier when a group is the whole block).  Block b
// takes every gridDim-th entry of each list.
template <class KT>
__device__ __forceinline__ void coop_networks(const Params& P, int p, const ListCounts& cur,
                                              typename KT::U* stage) {
  using U = typename KT::U;
  using G = SmallGroup<KT>;
  using CS = CoopShape<KT>;
  constexpr int T = kCoopThreads, W = CS::WARPS;
  constexpr int kMax = small_warp_max<KT, false>();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t cap = P.l.cap_run;
  for (uint32_t s = blockIdx.x * W + warp; s < min(cur.tiny, cap); s += gridDim.x * W) {
    const Run r = P.l.tiny[p][s];
    U* sx = stage + warp * kWarpSortMax;
    if (r.len <= 32) sort_run<KT, false, 1, 32>(P, r, lane, sx, nullptr, false);
    else if (r.len <= 64) sort_run<KT, false, 2, 32>(P, r, lane, sx, nullptr, false);
    else if (r.len <= 128) sort_run<KT, false, 4, 32>(P, r, lane, sx, nullptr, false);
    else sort_run<KT, false, 8, 32>(P, r, lane, sx, nullptr, false);
  }
  __syncthreads();
  for (uint32_t s = blockIdx.x * W + warp; s < min(cur.small, cap); s += gridDim.x * W) {
    const Run r = P.l.small[p][s];
    U* sw = stage + warp * CS::kWarpStage;
    if (r.len <= 512) group_sort_run<KT, 512 / 32, 32>(P, r, lane, sw);
    else if constexpr (kMax >= 1024) group_sort_run<KT, 1024 / 32, 32>(P, r, lane, sw);
  }
  __syncthreads();
  {
    constexpr int NG = T / G::T;
    const int g = tid / G::T, gt = tid % G::T;
    U* sw = stage + g * staging_entries<U, G::RMAX, G::T>();
    for (uint32_t s = blockIdx.x * NG + g; s < min(cur.group, cap); s += gridDim.x * NG) {
      const Run r = P.l.group[p][s];
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
    for (uint32_t s = blockIdx.x * NG + g; s < min(cur.big, cap); s += gridDim.x * NG) {
      const Run r = P.l.big[p][s];
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

// Bookkeeping of the large segments of parity p (the main loop's recursion): the pivot
// class of each is written now (at most kInlineFill keys) or queued on q's fill list,
// and both children, pivot class excluded (Sec. 2), go to the lists of q.
template <class KT>
__device__ __forceinline__ void coop_bookkeep(const Params& P, int p, int q, uint32_t count) {
  using U = typename KT::U;
  const int lane = threadIdx.x & 31;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x; base < count; base += stride) {
    const uint32_t s = base + threadIdx.x;
    const bool active = s < count;
    Seg sg{};
    int64_t nlt = 0, ngt = 0, neq = 0;
    if (active) {
      sg = P.l.large[p][s];
      const unsigned long long cur = P.l.cursor[p][s];
      nlt = (uint32_t)cur;
      ngt = (uint32_t)(cur >> 32);
      neq = sg.len - nlt - ngt;
    }
    unsigned long long moved = (unsigned long long)(nlt + ngt), eq = (unsigned long long)neq;
    for (int o = 16; o; o >>= 1) {
      moved += __shfl_xor_sync(~0u, moved, o);
      eq += __shfl_xor_sync(~0u, eq, o);
    }
    if (lane == 0) {
      atomicAdd(&P.ctrl->moved_keys, moved);
      atomicAdd(&P.ctrl->equal_keys, eq);
    }
    if (active && neq > 0 && neq <= kInlineFill) {
      U* fk = (U*)P.b.final_key + sg.off + nlt;
      for (int64_t j = 0; j < neq; ++j) fk[j] = (U)sg.pkey;
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
      if (lane == 31) fb = atomicAdd(&P.ctrl->lists[q].fill, v);
      fb = __shfl_sync(~0u, fb, 31);
      if (fills) {
        const unsigned long long old = fb + v - own;
        const uint32_t slot = (uint32_t)old;
        if (slot < P.l.cap_fill) {
          Fill f;
          f.off = sg.off + nlt; f.len = neq; f.pkey = sg.pkey; f.pval = 0;
          f.tile0 = (uint32_t)(old >> 32);
          P.l.fill[q][slot] = f;
        } else {
          atomicExch(&P.ctrl->status, kStatusOverflow);
        }
      }
    }
    route_warp<KT, false>(P, q, active, sg.off, nlt, sg.parity ^ 1, sg.depth + 1);
    route_warp<KT, false>(P, q, active, sg.off + sg.len - ngt, ngt, sg.parity ^ 1, sg.depth + 1);
  }
}

// The cooperative sort of keys[0, n) (key-only).  Launched with every block resident;
// the host has cleared the control block.
template <class KT>
__global__ void __launch_bounds__(kCoopThreads, 2) k_coop_sort(Params P, int64_t n, int max_levels) {
  using U = typename KT::U;
  extern __shared__ __align__(16) unsigned char coop_smem[];
  U* stage = reinterpret_cast<U*>(coop_smem);
  __shared__ PivotSmem<KT, false> psm;
  __shared__ uint32_t s_wcnt[CoopShape<KT>::WARPS];
  __shared__ unsigned long long s_base;
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
    const int p = level & 1, q = p ^ 1;
    // Every block reads the same counts: nothing writes them between the last barrier
    // and the clear of lists[q] below (a different entry).
    const volatile ListCounts* vl = &c->lists[p];
    ListCounts cur;
    cur.large = vl->large; cur.fill = vl->fill; cur.large_keys = vl->large_keys;
    cur.small = vl->small; cur.tiny = vl->tiny; cur.todo = vl->todo; cur.local = vl->local;
    cur.group = vl->group; cur.big = vl->big;
    const uint32_t nlarge = min((uint32_t)cur.large, P.l.cap_large);
    const uint32_t ntiles = nlarge ? (uint32_t)(cur.large >> 32) : 0u;
    if (*(volatile int*)&c->status != 0) break;
    if (!(nlarge | cur.tiny | cur.small | cur.group | cur.big | (uint32_t)cur.fill)) break;
    if (level > max_levels) {
      if (lead) atomicExch(&c->status, kStatusOverflow);
      break;
    }
    if (cur.todo && nlarge) {   // sample pivots (sqrt(n) rule) and depth-limit fallbacks
      pivot_pass<KT, false>(P, p, psm);
      if (!coop_grid_sync(c, P.wait_limit, &s_ok)) return;
    }
    if (lead) clear_counts(&c->lists[q]);   // last read by the previous bookkeeping
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x)
      coop_tile<KT>(P, p, t, nlarge, stage, s_wcnt, &s_base, &s_idx);
    __syncthreads();   // the tiles' staging area becomes the networks'
    coop_networks<KT>(P, p, cur, stage);
    coop_fills<KT>(P, p, cur.fill, &s_idx);
    if (!coop_grid_sync(c, P.wait_limit, &s_ok)) return;
    coop_bookkeep<KT>(P, p, q, nlarge);
    if (lead) {
      if (nlarge) {
        c->levels_run += 1;
        c->active_total += cur.large_keys;
      }
      c->small_runs += cur.tiny + cur.small + cur.group + cur.big;
    }
    if (!coop_grid_sync(c, P.wait_limit, &s_ok)) return;
  }
  if (lead) c->level = level;
}

}  // namespace bqs

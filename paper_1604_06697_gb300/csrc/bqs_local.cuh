// Single-block local partitioning: the bottom partition levels of the recursion inside
// shared memory.
//
// One thread block takes a whole segment of at most L keys (the `local` list), loads it
// once into a shared-memory buffer and keeps applying the block partition step of
// Sec. 3 to all of its unfinished sub-segments at once, ping-ponging between two
// shared-memory buffers, until every sub-segment is short enough for a sorting network
// (at most the small-segment cutoff).  After each level the pivot classes are written
// to the final buffer (the pivot value, as everywhere).  The finished sub-segments
// either are written back to the segment's range in HBM and appended to the next
// level's network lists, or (SORT, key-only sorts) stay in shared memory and are
// sorted there by the warp-group networks once the block's levels are done, straight
// into the final buffer: the single-block sort of the segment (partition levels and
// networks) then costs one HBM read and one write per key in total.  The recursion is
// the same as on the global levels (the same pivot rules, three-way split, pivot class
// excluded from both sides).
#pragma once

#include "bqs_small.cuh"

namespace bqs {

constexpr int kLocalMaxAct = 64;    // active sub-segments per level (> L / kWarpSortMax)
constexpr int kLocalMaxLeaf = 128;  // finished sub-segments per level (2 per active one)
constexpr int kLocalChunk = 256;    // keys per warp work item (32 lanes x 8)
constexpr int kLocalSortCap = 128;  // sub-segments one block sorts itself (SORT); more
                                    // go back to HBM and the network kernels

struct SubSeg {
  int begin;   // offset in the block's segment
  int len;
  int buf;     // shared-memory buffer holding its keys
  int depth;   // partition levels above it
};

// Shared memory: key buffers 0 and 1 (L keys each; with SORT buffer 1 also holds the
// staging rows of the block's network groups), then payload buffers 0 and 1.
template <class KT, bool PAIRS, int L, int T, bool SORT>
struct LocalShape {
  using U = typename KT::U;
  using G = SmallGroup<KT>;
  static constexpr int kStageBig = (T / G::TBIG) * staging_entries<U, G::RMAX, G::TBIG>();
  static constexpr int kStageSmall = (T / G::T) * staging_entries<U, G::RMAX, G::T>();
  static constexpr int kEntries1 =
      !SORT ? L : (L > kStageBig ? (L > kStageSmall ? L : kStageSmall)
                                 : (kStageBig > kStageSmall ? kStageBig : kStageSmall));
  static constexpr size_t kbuf = (size_t)L * sizeof(U);
  static constexpr size_t kbuf1 = (size_t)kEntries1 * sizeof(U);
  static constexpr size_t vbuf = PAIRS ? (size_t)L * 4 : 0;
  static constexpr size_t smem = kbuf + kbuf1 + 2 * vbuf;
};

// The leaves one block sorts itself (SORT): first those above kMaxSmall keys, one
// group of SmallGroup::TBIG threads each, then the others, one group of SmallGroup::T
// threads each with the smallest of RMAX/4, RMAX/2, RMAX keys per thread that holds
// the leaf.  Every leaf is in key buffer `kb0`; `stage` (key buffer 1) holds the
// groups' staging rows.  Groups take leaves round-robin; every decision below is
// uniform within a group, so its named barriers line up.
template <class KT, int T>
__device__ __forceinline__ void local_sort_leaves(const SubSeg* leaves, int nleaves,
                                                  const typename KT::U* kb0,
                                                  typename KT::U* stage, typename KT::U* fk,
                                                  int tid) {
  using U = typename KT::U;
  using G = SmallGroup<KT>;
  {
    constexpr int NG = T / G::TBIG;
    const int g = tid / G::TBIG, gt = tid % G::TBIG;
    U* sw = stage + g * staging_entries<U, G::RMAX, G::TBIG>();
    for (int f = 0, k = 0; f < nleaves; ++f) {
      const SubSeg a = leaves[f];
      if (a.len <= kMaxSmall) continue;
      if (k++ % NG != g) continue;
      // (a group that is the whole block, 64-bit keys, takes the block barrier)
      group_sort_keys<KT, G::RMAX, G::TBIG, (G::TBIG < T)>(kb0 + a.begin, fk + a.begin, a.len, gt, sw);
    }
  }
  __syncthreads();   // the staging rows change owners
  {
    constexpr int NG = T / G::T;
    const int g = tid / G::T, gt = tid % G::T;
    U* sw = stage + g * staging_entries<U, G::RMAX, G::T>();
    for (int f = 0, k = 0; f < nleaves; ++f) {
      const SubSeg a = leaves[f];
      if (a.len > kMaxSmall) continue;
      if (k++ % NG != g) continue;
      if (a.len <= (G::RMAX / 4) * G::T)
        group_sort_keys<KT, G::RMAX / 4, G::T, true>(kb0 + a.begin, fk + a.begin, a.len, gt, sw);
      else if (a.len <= (G::RMAX / 2) * G::T)
        group_sort_keys<KT, G::RMAX / 2, G::T, true>(kb0 + a.begin, fk + a.begin, a.len, gt, sw);
      else
        group_sort_keys<KT, G::RMAX, G::T, true>(kb0 + a.begin, fk + a.begin, a.len, gt, sw);
    }
  }
}

template <class KT, bool PAIRS, int L, int T, bool SORT>
__global__ void __launch_bounds__(T, SORT ? 2 : 3) k_local_partition(Params P, int p) {
  using U = typename KT::U;
  using S = LocalShape<KT, PAIRS, L, T, SORT>;
  using E = Elem<KT, PAIRS>;
  constexpr int WARPS = T / 32;
  constexpr int KPL = kLocalChunk / 32;
  constexpr int KPT = L / T;                   // keys per thread of the segment's load
  static_assert(L % T == 0, "whole loads per thread");
  static_assert(!(SORT && PAIRS), "the block's own networks are key-only");
  static_assert(L / (kWarpSortMax + 1) + 1 <= kLocalMaxAct, "active list capacity");
  static_assert(2 * kLocalMaxAct <= kLocalMaxLeaf, "leaf list capacity");
  static_assert(L < 65536, "packed per-sub-segment counts");

  p = level_parity(P, p);
  const int q = p ^ 1;
  extern __shared__ __align__(16) unsigned char smem[];
  // buffer b: keys at smem + b*kbuf, payloads at smem + kbuf + kbuf1 + b*vbuf
  auto kb = [&](int b) { return reinterpret_cast<U*>(smem + (size_t)b * S::kbuf); };
  auto vb = [&](int b) { return reinterpret_cast<uint32_t*>(smem + S::kbuf + S::kbuf1 + (size_t)b * S::vbuf); };
  __shared__ SubSeg s_act[2][kLocalMaxAct];
  __shared__ U s_pk[kLocalMaxAct];            // pivot of each active sub-segment (raw bits)
  __shared__ uint32_t s_pv[kLocalMaxAct];
  __shared__ uint32_t s_vstart[kLocalMaxAct + 1];  // work-item starts, padded to kLocalChunk
  __shared__ uint32_t s_cnt[kLocalMaxAct];    // (#<) | (#>) << 16 claimed so far
  __shared__ SubSeg s_leaf[kLocalMaxLeaf];    // finished this level
  __shared__ int s_fill[kLocalMaxAct][2];     // pivot class: begin, length
  __shared__ int s_nact[2], s_nleaf;
  __shared__ SubSeg s_done[SORT ? kLocalSortCap : 1];   // leaves this block sorts (SORT)
  __shared__ int s_ndone;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cap = SORT ? min(P.local_sort, kLocalSortCap) : 0;   // leaves sorted here
  const unsigned int count = min(P.ctrl->lists[p].local, P.l.cap_run);
  U* fk = (U*)P.b.final_key;
  uint32_t* fv = P.b.final_val;

  for (unsigned int r = blockIdx.x; r < count; r += gridDim.x) {
    const Run run = P.l.local[p][r];
    const int len = (int)run.len;
    const int X = run.parity;                  // leaves go back to the run's own range
    U* gk = (U*)P.b.key[X] + run.off;
    uint32_t* gv = PAIRS ? P.b.val[X] + run.off : nullptr;
    {
      // All of a thread's loads are issued before its first shared-memory store.
      U* k0 = kb(0);
      U kv[KPT];
#pragma unroll
      for (int i = 0; i < KPT; ++i) {
        const int e = i * T + tid;
        kv[i] = e < len ? gk[e] : U(0);
      }
#pragma unroll
      for (int i = 0; i < KPT; ++i) {
        const int e = i * T + tid;
        if (e < len) k0[e] = kv[i];
      }
      if constexpr (PAIRS) {
        uint32_t* v0 = vb(0);
#pragma unroll
        for (int i = 0; i < KPT; ++i) {
          const int e = i * T + tid;
          kv[i] = e < len ? (U)gv[e] : U(0);
        }
#pragma unroll
        for (int i = 0; i < KPT; ++i) {
          const int e = i * T + tid;
          if (e < len) v0[e] = (uint32_t)kv[i];
        }
      }
    }
    if (tid == 0) {
      s_nact[0] = 1;
      s_nact[1] = 0;
      s_act[0][0] = SubSeg{0, len, 0, run.pad};
      s_ndone = 0;
    }
    __syncthreads();

    for (int cur = 0;; cur ^= 1) {
      const int nact = s_nact[cur];
      if (nact == 0) {
        if constexpr (SORT) {
          // Leaves in buffer 1 move to buffer 0, which then holds every leaf; buffer 1
          // becomes the networks' staging rows.
          const int nd = min(s_ndone, cap);
          for (int f = warp; f < nd; f += WARPS) {
            const SubSeg a = s_done[f];
            if (a.buf == 1)
              for (int i = lane; i < a.len; i += 32) kb(0)[a.begin + i] = kb(1)[a.begin + i];
          }
          __syncthreads();
          local_sort_leaves<KT, T>(s_done, nd, kb(0), kb(1), fk + run.off, tid);
          __syncthreads();   // shared memory is reused by the next run
        }
        break;
      }

      // Pivots (the depth-limit fallback: midpoint of the ord-key range, then of the
      // payload range, as in k_pivot) and work-item starts.
      if (tid < nact) {
        const SubSeg a = s_act[cur][tid];
        const U* kk = kb(a.buf) + a.begin;
        const uint32_t* vv = vb(a.buf) + a.begin;
        E piv;
        if (a.depth < P.depth_limit) {
          piv = rule_pivot<KT, PAIRS>(kk, vv, 0, a.len, P.pivot_rule);   // as on global levels
        } else {
          U kmin = ~U(0), kmax = 0;
          for (int i = 0; i < a.len; ++i) {
            const U k = KT::ord(kk[i]);
            kmin = k < kmin ? k : kmin;
            kmax = k > kmax ? k : kmax;
          }
          piv.k = kmin + (kmax - kmin) / 2;
          piv.v = 0xFFFFFFFFu;
          if (PAIRS && kmin == kmax) {
            uint32_t vmin = 0xFFFFFFFFu, vmax = 0;
            for (int i = 0; i < a.len; ++i) {
              vmin = min(vmin, vv[i]);
              vmax = max(vmax, vv[i]);
            }
            piv.v = vmin + (vmax - vmin) / 2;
          }
          atomicAdd(&P.ctrl->fallbacks, 1ull);
        }
        s_pk[tid] = KT::unord(piv.k);
        s_pv[tid] = piv.v;
        s_cnt[tid] = 0;
      }
      if (warp == 0) {   // exclusive scan of the padded lengths (4 entries per lane)
        uint32_t v[4], sum = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int j = lane * 4 + i;
          v[i] = j < nact ? (uint32_t)((s_act[cur][j].len + kLocalChunk - 1) / kLocalChunk) * kLocalChunk : 0u;
          sum += v[i];
        }
        uint32_t incl = sum;
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(~0u, incl, o);
          if (lane >= o) incl += y;
        }
        uint32_t run_ = incl - sum;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int j = lane * 4 + i;
          if (j <= nact) s_vstart[j] = run_;
          run_ += v[i];
        }
        if (lane == 0) { s_nact[cur ^ 1] = 0; s_nleaf = 0; }
      }
      __syncthreads();

      // Partition pass over all active sub-segments (Algorithm 3 per 256-key work
      // item): one warp per item, outcomes counted per lane, one shared-memory atomic
      // per item reserves both runs.
      const int nitems = (int)(s_vstart[nact] / kLocalChunk);
      for (int it = warp; it < nitems; it += WARPS) {
        const uint32_t v0 = (uint32_t)it * kLocalChunk;
        int lo = 0, hi = nact;                         // last j with s_vstart[j] <= v0
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (s_vstart[mid] <= v0) lo = mid; else hi = mid;
        }
        const int j = lo;
        const SubSeg a = s_act[cur][j];
        const int base = (int)(v0 - s_vstart[j]);
        const U* src = kb(a.buf) + a.begin;
        const uint32_t* vsrc = vb(a.buf) + a.begin;
        U* dst = kb(a.buf ^ 1) + a.begin;
        uint32_t* vdst = vb(a.buf ^ 1) + a.begin;
        const U pk = s_pk[j];
        const U pko = KT::ord(pk);
        const uint32_t pv = s_pv[j];
        U key[KPL];
        uint32_t val[PAIRS ? KPL : 1];
        uint32_t cl = 0, cg = 0;
#pragma unroll
        for (int k = 0; k < KPL; ++k) {
          const int idx = base + k * 32 + lane;
          const bool valid = idx < a.len;
          key[k] = valid ? src[idx] : pk;          // outside: counts as equal
          if constexpr (PAIRS) val[k] = valid ? vsrc[idx] : pv;
          const U ko = KT::ord(key[k]);
          const uint32_t vv = PAIRS ? val[k] : 0u;
          cl += elem_less<PAIRS>(ko, vv, pko, pv);
          cg += elem_less<PAIRS>(pko, pv, ko, vv);
        }
        const uint32_t own = cl | (cg << 16);
        uint32_t incl = own;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(~0u, incl, o);
          if (lane >= o) incl += y;
        }
        uint32_t wb = 0;
        if (lane == 31) wb = atomicAdd(&s_cnt[j], incl);   // both runs in one atomic
        wb = __shfl_sync(~0u, wb, 31);
        const uint32_t excl = incl - own;
        int pl = (int)((wb & 0xFFFF) + (excl & 0xFFFF));
        int pg = a.len - (int)((wb >> 16) + (excl >> 16)) - (int)cg;
#pragma unroll
        for (int k = 0; k < KPL; ++k) {
          const U ko = KT::ord(key[k]);
          const uint32_t vv = PAIRS ? val[k] : 0u;
          const bool l = elem_less<PAIRS>(ko, vv, pko, pv);
          const bool g = elem_less<PAIRS>(pko, pv, ko, vv);
          if (l) {
            dst[pl] = key[k];
            if constexpr (PAIRS) vdst[pl] = val[k];
          }
          if (g) {
            dst[pg] = key[k];
            if constexpr (PAIRS) vdst[pg] = val[k];
          }
          pl += l;
          pg += g;
        }
      }
      __syncthreads();

      // Children: sub-segments above the small-segment cutoff stay active, the others
      // are finished here; the pivot class is final.
      if (tid < nact) {
        const SubSeg a = s_act[cur][tid];
        const int nlt = (int)(s_cnt[tid] & 0xFFFF), ngt = (int)(s_cnt[tid] >> 16);
        s_fill[tid][0] = a.begin + nlt;
        s_fill[tid][1] = a.len - nlt - ngt;
        const SubSeg kids[2] = {SubSeg{a.begin, nlt, a.buf ^ 1, a.depth + 1},
                                SubSeg{a.begin + a.len - ngt, ngt, a.buf ^ 1, a.depth + 1}};
        for (int c = 0; c < 2; ++c) {
          if (kids[c].len == 0) continue;
          if (kids[c].len <= P.small_cutoff) {
            int d = cap;
            if constexpr (SORT) d = atomicAdd(&s_ndone, 1);
            if (d < cap) s_done[d] = kids[c];                      // sorted here at the end
            else s_leaf[atomicAdd(&s_nleaf, 1)] = kids[c];          // back to HBM
          } else
            s_act[cur ^ 1][atomicAdd(&s_nact[cur ^ 1], 1)] = kids[c];
        }
      }
      __syncthreads();

      // Finished keys leave shared memory: pivot classes to the final buffer, finished
      // sub-segments back to the run's range (one warp per sub-segment, coalesced).
      const int nleaf = s_nleaf;
      for (int f = warp; f < nact + nleaf; f += WARPS) {
        if (f < nact) {
          const int b = s_fill[f][0], n = s_fill[f][1];
          const U pk = s_pk[f];
          const uint32_t pv = s_pv[f];
          for (int i = lane; i < n; i += 32) {
            fk[run.off + b + i] = pk;
            if constexpr (PAIRS) fv[run.off + b + i] = pv;
          }
        } else {
          const SubSeg a = s_leaf[f - nact];
          const U* ks = kb(a.buf) + a.begin;
          const uint32_t* vs = vb(a.buf) + a.begin;
          for (int i = lane; i < a.len; i += 32) {
            gk[a.begin + i] = ks[i];
            if constexpr (PAIRS) gv[a.begin + i] = vs[i];
          }
        }
      }
      __syncthreads();   // the leaves' keys are in HBM before anyone routes them

      // Appended to the network lists of the next level (warp-aggregated, like every
      // child segment); their keys were counted when the run was routed here.
      for (int base = warp * 32; base < nleaf; base += WARPS * 32) {
        const int f = base + lane;
        const bool has = f < nleaf;
        const SubSeg a = has ? s_leaf[f] : SubSeg{0, 0, 0, 0};
        route_warp<KT, PAIRS>(P, q, has, run.off + a.begin, a.len, X, a.depth, false);
      }
      __syncthreads();
    }
  }
}

}  // namespace bqs

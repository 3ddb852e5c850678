// Single-block local sort: the bottom levels of the recursion inside shared memory.
//
// One thread block takes a whole segment of at most L keys, loads it once into a
// shared-memory buffer, and keeps applying the block partition step of Sec. 3 to all
// of its unfinished sub-segments at once, ping-ponging between two shared-memory
// buffers, until every sub-segment has at most kLocalLeaf keys.  Those leaves are
// finished by the warp sorting network of bqs_small.cuh (the stand-in for the paper's
// Insertionsort), and the assembled segment is written to HBM once.  The result is the
// same Quicksort recursion as the global levels (median pivots, three-way split, pivot
// class excluded from both sides), with one HBM read and one write per key instead of
// one per level.
#pragma once

#include "bqs_small.cuh"

namespace bqs {

constexpr int kLocalMaxAct = 128;  // unfinished sub-segments per level (> L / kLocalLeaf)
constexpr int kLocalChunk = 256;   // keys per warp work item (32 lanes x 8)
constexpr int kLocalLeaf = 256;    // sub-segments up to this length go to a warp network

struct SubSeg {
  int begin;   // offset in the block's segment
  int len;
  int buf;     // shared-memory buffer holding its keys
  int depth;   // local partition levels above it
};

template <class KT, bool PAIRS, int L>
struct LocalShape {
  using U = typename KT::U;
  static constexpr size_t kbuf = (size_t)L * sizeof(U);
  static constexpr size_t vbuf = PAIRS ? (size_t)L * 4 : 0;
  static constexpr size_t smem = 2 * (kbuf + vbuf);
};

// Sorts len <= 32*R entries at src[0, len) (shared memory, raw keys) into dst[0, len)
// with one warp; src and dst may be the same.
template <class KT, bool PAIRS, int R>
__device__ __forceinline__ void warp_sort_smem(const typename KT::U* src, const uint32_t* vsrc,
                                               typename KT::U* dst, uint32_t* vdst, int len,
                                               int lane) {
  using U = typename KT::U;
  U x[R];
  uint32_t y[R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int e = lane * R + i;
    x[i] = e < len ? KT::ord(src[e]) : ~U(0);
    y[i] = PAIRS ? (e < len ? vsrc[e] : 0xFFFFFFFFu) : 0u;
  }
  __syncwarp();
  net_sort<PAIRS, R, 32>(x, y, lane, (U*)nullptr, (uint32_t*)nullptr);
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int e = lane * R + i;
    if (e < len) {
      dst[e] = KT::unord(x[i]);
      if constexpr (PAIRS) vdst[e] = y[i];
    }
  }
  __syncwarp();
}

template <class KT, bool PAIRS>
__device__ __forceinline__ void warp_sort_leaf(const typename KT::U* src, const uint32_t* vsrc,
                                               typename KT::U* dst, uint32_t* vdst, int len,
                                               int lane) {
  if (len <= 32) warp_sort_smem<KT, PAIRS, 1>(src, vsrc, dst, vdst, len, lane);
  else if (len <= 64) warp_sort_smem<KT, PAIRS, 2>(src, vsrc, dst, vdst, len, lane);
  else if (len <= 128) warp_sort_smem<KT, PAIRS, 4>(src, vsrc, dst, vdst, len, lane);
  else warp_sort_smem<KT, PAIRS, 8>(src, vsrc, dst, vdst, len, lane);
}

// Leaves are recorded as begin | (len - 1) << 15 | buffer << 24 (begin < 2^15, len <= 256).
__device__ __forceinline__ uint32_t pack_leaf(int begin, int len, int buf) {
  return (uint32_t)begin | ((uint32_t)(len - 1) << 15) | ((uint32_t)buf << 24);
}

template <class KT, bool PAIRS, int L, int T>
__global__ void __launch_bounds__(T) k_local_sort(Params P, int p) {
  using U = typename KT::U;
  p = level_parity(P, p);
  using S = LocalShape<KT, PAIRS, L>;
  using E = Elem<KT, PAIRS>;
  constexpr int WARPS = T / 32;
  constexpr int KPL = kLocalChunk / 32;
  constexpr int MAXLEAF = 2048;
  static_assert(L / (kLocalLeaf + 1) + 1 <= kLocalMaxAct, "active list capacity");
  static_assert(L <= 32768 && kLocalLeaf <= 256, "leaf record packing");

  extern __shared__ __align__(16) unsigned char smem[];
  // buffer b: keys at smem + b*kbuf, payloads at smem + 2*kbuf + b*vbuf
  auto kb = [&](int b) { return reinterpret_cast<U*>(smem + (size_t)b * S::kbuf); };
  auto vb = [&](int b) { return reinterpret_cast<uint32_t*>(smem + 2 * S::kbuf + (size_t)b * S::vbuf); };
  __shared__ SubSeg s_act[2][kLocalMaxAct];
  __shared__ U s_pk[kLocalMaxAct];            // pivot of each active sub-segment (raw bits)
  __shared__ uint32_t s_pv[kLocalMaxAct];
  __shared__ uint32_t s_vstart[kLocalMaxAct + 1];  // work-item starts, padded to kLocalChunk
  __shared__ uint32_t s_cnt[kLocalMaxAct];    // (#<) | (#>) << 16 claimed so far
  __shared__ uint32_t s_leaf[MAXLEAF];
  __shared__ int s_nact[2], s_nleaf;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned int count = min(P.ctrl->lists[p].local, P.l.cap_run);
  const int depth_cap = 2 * (31 - __clz(L)) + 8;   // local Introsort-style limit

  // Sorts every recorded leaf into buffer 0, warps taking leaves round-robin.
  auto flush_leaves = [&]() {
    const int nl = s_nleaf;
    for (int f = warp; f < nl; f += WARPS) {
      const uint32_t q = s_leaf[f];
      const int b = (int)(q & 0x7FFF), ln = (int)((q >> 15) & 0x1FF) + 1, bf = (int)(q >> 24);
      warp_sort_leaf<KT, PAIRS>(kb(bf) + b, vb(bf) + b, kb(0) + b, vb(0) + b, ln, lane);
    }
  };

  for (unsigned int r = blockIdx.x; r < count; r += gridDim.x) {
    const Run run = P.l.local[p][r];
    const int len = (int)run.len;
    {
      const U* g = (const U*)P.b.key[run.parity] + run.off;
      const uint32_t* gv = PAIRS ? P.b.val[run.parity] + run.off : nullptr;
      U* k0 = kb(0);
      uint32_t* v0 = vb(0);
      for (int i = tid; i < len; i += T) {
        k0[i] = g[i];
        if constexpr (PAIRS) v0[i] = gv[i];
      }
    }
    if (tid == 0) {
      s_nleaf = 0;
      s_nact[1] = 0;
      if (len <= kLocalLeaf) {
        s_nact[0] = 0;
        s_leaf[0] = pack_leaf(0, len, 0);
        s_nleaf = 1;
      } else {
        s_nact[0] = 1;
        s_act[0][0] = SubSeg{0, len, 0, 0};
      }
    }
    __syncthreads();

    for (int cur = 0;; cur ^= 1) {
      const int nact = s_nact[cur];
      if (nact == 0) break;
      // Keep room for this level's leaves (at most two per active sub-segment).
      if (s_nleaf + 2 * nact > MAXLEAF) {
        flush_leaves();
        __syncthreads();
        if (tid == 0) s_nleaf = 0;
      }

      // Pivots (median of three medians of three of nine spaced keys; the midpoint of
      // the ord-key range past the local depth cap) and work-item starts.
      if (tid < nact) {
        const SubSeg a = s_act[cur][tid];
        const U* kk = kb(a.buf) + a.begin;
        const uint32_t* vv = vb(a.buf) + a.begin;
        E piv;
        if (a.depth < depth_cap) {
          E m[3];
          for (int g = 0; g < 3; ++g)
            m[g] = median3<KT, PAIRS>(
                load_elem<KT, PAIRS>(kk, vv, ((2 * (3 * g + 0) + 1) * a.len) / 18),
                load_elem<KT, PAIRS>(kk, vv, ((2 * (3 * g + 1) + 1) * a.len) / 18),
                load_elem<KT, PAIRS>(kk, vv, ((2 * (3 * g + 2) + 1) * a.len) / 18));
          piv = median3<KT, PAIRS>(m[0], m[1], m[2]);
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
        if (lane == 0) s_nact[cur ^ 1] = 0;
      }
      __syncthreads();

      // Partition pass over all active sub-segments: one warp per 256-key work item.
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

      // Children of every active sub-segment; the pivot class is final: it is written
      // to buffer 0 right away (usually a single key).
      if (tid < nact) {
        const SubSeg a = s_act[cur][tid];
        const int nlt = (int)(s_cnt[tid] & 0xFFFF), ngt = (int)(s_cnt[tid] >> 16);
        const int neq = a.len - nlt - ngt;
        U* k0 = kb(0) + a.begin + nlt;
        uint32_t* v0 = vb(0) + a.begin + nlt;
        for (int i = 0; i < neq; ++i) {
          k0[i] = s_pk[tid];
          if constexpr (PAIRS) v0[i] = s_pv[tid];
        }
        const SubSeg kids[2] = {SubSeg{a.begin, nlt, a.buf ^ 1, a.depth + 1},
                                SubSeg{a.begin + a.len - ngt, ngt, a.buf ^ 1, a.depth + 1}};
        for (int c = 0; c < 2; ++c) {
          if (kids[c].len == 0) continue;
          if (kids[c].len <= kLocalLeaf)
            s_leaf[atomicAdd(&s_nleaf, 1)] = pack_leaf(kids[c].begin, kids[c].len, kids[c].buf);
          else
            s_act[cur ^ 1][atomicAdd(&s_nact[cur ^ 1], 1)] = kids[c];
        }
      }
      __syncthreads();
    }
    flush_leaves();
    __syncthreads();

    // The assembled segment goes to the final buffer once.
    {
      U* g = (U*)P.b.final_key + run.off;
      uint32_t* gv = PAIRS ? P.b.final_val + run.off : nullptr;
      const U* k0 = kb(0);
      const uint32_t* v0 = vb(0);
      for (int i = tid; i < len; i += T) {
        g[i] = k0[i];
        if constexpr (PAIRS) gv[i] = v0[i];
      }
    }
    __syncthreads();
  }
}

}  // namespace bqs

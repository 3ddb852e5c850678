// TMA-fed persistent variant of the block partition step (sm_90+ bulk copies, mbarriers).
//
// Each thread block owns a contiguous range of the level's tiles and runs a STAGES-deep
// ring of shared-memory tile buffers: thread 0 issues one cp.async.bulk (global ->
// shared, completion counted on an mbarrier) per tile and per array, STAGES-1 tiles
// ahead of the tile being partitioned, so HBM latency is hidden with one or two blocks
// per SM instead of by occupancy.  The partition of a tile is the same Algorithm 3 step
// as k_partition: compare, outcome bits in registers, warp totals, one packed atomic
// per tile, staging in output order, coalesced write-out.
#pragma once

#include "bqs_kernels.cuh"

namespace bqs {

// ---- PTX wrappers (bulk copy + mbarrier) -------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;"
               ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Returns true when the phase with the given parity has completed.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  return done != 0;
}

__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_u32(dst_smem)), "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

// Bounded wait on an mbarrier phase: gives up after `limit` polls (2^26 by default,
// seconds), records a timeout in the device status word and reports failure to the
// caller, which then leaves the kernel instead of hanging.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, Ctrl* ctrl,
                                                  uint32_t limit) {
  for (uint32_t it = 0; it < limit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (it > 64) __nanosleep(32);
  }
  atomicExch(&ctrl->status, kStatusTimeout);
  return false;
}

// Comparable image of a raw key: signed integers compare natively, float64 through ord.
template <class KT> struct Cmp;
template <> struct Cmp<KeyI32> {
  using T = int32_t;
  __device__ static __forceinline__ T of(uint32_t x) { return (int32_t)x; }
};
template <> struct Cmp<KeyI64> {
  using T = int64_t;
  __device__ static __forceinline__ T of(uint64_t x) { return (int64_t)x; }
};
template <> struct Cmp<KeyF64> {
  using T = uint64_t;
  __device__ static __forceinline__ T of(uint64_t x) { return KeyF64::ord(x); }
};

template <bool PAIRS, class T>
__device__ __forceinline__ bool cmp_less(T ka, uint32_t va, T kb, uint32_t vb) {
  if constexpr (PAIRS) return ka < kb || (ka == kb && va < vb);
  else return ka < kb;
}

// Per-tile description kept in shared memory for the tiles of the current chunk.
struct TileInfo {
  int64_t off;     // segment start
  int64_t len;     // segment length
  uint64_t pkey;   // pivot (raw bits)
  uint32_t seg;    // index in the level's list (cursor slot)
  uint32_t pval;   // pivot payload
  int32_t parity;  // source buffer
  int32_t pad;     // the segment's depth
};

template <class KT, bool PAIRS, int THREADS, int KPT, int STAGES, int CHUNK_ = 256>
struct TmaShape {
  using U = typename KT::U;
  static constexpr int TILE = THREADS * KPT;
  static constexpr int CHUNK = CHUNK_;    // tiles whose descriptors are looked up at once
  static constexpr size_t in_bytes = (size_t)STAGES * TILE * sizeof(U);
  static constexpr size_t vin_bytes = PAIRS ? (size_t)STAGES * TILE * 4 : 0;
  static constexpr size_t out_bytes = (size_t)TILE * sizeof(U);
  static constexpr size_t vout_bytes = PAIRS ? (size_t)TILE * 4 : 0;
  static constexpr size_t info_bytes = (size_t)2 * CHUNK * sizeof(TileInfo);
  static constexpr size_t smem = in_bytes + vin_bytes + out_bytes + vout_bytes + info_bytes;
};

// FUSED: the instantiation for levels of few tiles per block, which also does the
// bookkeeping of each segment (see the end of the tile loop).
template <class KT, bool PAIRS, int THREADS, int KPT, int STAGES, int CHUNK_ = 256, int MINB = 1,
          bool FUSED = false>
__global__ void __launch_bounds__(THREADS, MINB) k_partition_tma(Params P) {
  using U = typename KT::U;
  using S = TmaShape<KT, PAIRS, THREADS, KPT, STAGES, CHUNK_>;
  using CT = typename Cmp<KT>::T;
  constexpr int TILE = S::TILE;
  constexpr int VEC = 16 / sizeof(U);
  constexpr int NV = KPT / VEC;
  constexpr int WARPS = THREADS / 32;
  constexpr int CHUNK = S::CHUNK;
  static_assert(KPT % VEC == 0 && KPT <= 32 && TILE <= 32768, "tile shape");
  static_assert(THREADS >= CHUNK && STAGES <= CHUNK, "descriptor chunking");
  static_assert(S::smem + 1024 <= 227 * 1024, "shared memory per block");

  extern __shared__ __align__(128) unsigned char smem[];
  U* s_in = reinterpret_cast<U*>(smem);
  uint32_t* s_vin = reinterpret_cast<uint32_t*>(smem + S::in_bytes);
  U* s_out = reinterpret_cast<U*>(smem + S::in_bytes + S::vin_bytes);
  uint32_t* s_vout = reinterpret_cast<uint32_t*>(smem + S::in_bytes + S::vin_bytes + S::out_bytes);
  TileInfo* s_info = reinterpret_cast<TileInfo*>(smem + S::in_bytes + S::vin_bytes + S::out_bytes +
                                                 S::vout_bytes);
  __shared__ __align__(8) uint64_t s_bar[STAGES];
  __shared__ uint32_t s_wcnt[WARPS];
  __shared__ unsigned long long s_base;
  __shared__ int s_abort;
  __shared__ uint32_t s_done_seg;   // fused bookkeeping: segment whose last tile this was
  __shared__ unsigned long long s_done_word;   // ... and its completion word
  __shared__ int s_copy;            // fused bookkeeping: the level's last segment

  // Launched as a programmatic dependent of the stream's previous kernel (deep host
  // loop), the block may start before that kernel has finished: it waits for it (and
  // its memory) here, and lets the next level's launch begin.  Both are no-ops
  // otherwise.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int pp = level_parity(P, P.p);
  // The lists this level's bookkeeping fills (after this kernel) start empty.  With the
  // bookkeeping fused into this kernel the previous level's last bookkeeping (or the
  // host) has emptied them already: other blocks may append to them at any time.
  if (!FUSED && blockIdx.x == 0 && threadIdx.x == 0) clear_counts(&P.ctrl->lists[pp ^ 1]);
  const unsigned long long lc = P.ctrl->lists[pp].large;
  const uint32_t nseg = min((uint32_t)lc, P.l.cap_large), ntiles = (uint32_t)(lc >> 32);
  const Seg* __restrict__ segs = P.l.large[pp];
  unsigned long long* cursor = P.l.cursor[pp];
  const int64_t n_total = P.n_keys;

  // Contiguous tile range of this block.
  const uint32_t t_begin = (uint32_t)(((uint64_t)ntiles * blockIdx.x) / gridDim.x);
  const uint32_t t_end = (uint32_t)(((uint64_t)ntiles * (blockIdx.x + 1)) / gridDim.x);
  const uint32_t count = t_end - t_begin;
  if (count == 0) return;

  // First tiles of the level's segments in shared memory (the staging buffer, unused
  // before the first tile) when there are between 8 and kTable of them, so that the
  // descriptor lookups before the tile loop search there instead of chaining global
  // loads.
  constexpr uint32_t kTable = (uint32_t)(S::out_bytes / sizeof(uint32_t));
  const bool table = nseg >= 8 && nseg <= kTable;
  const uint32_t* s_t0 = reinterpret_cast<const uint32_t*>(s_out);

  // Descriptors of tiles [t_begin + c*CHUNK, +CHUNK) into slot c&1: one binary search
  // per thread, then the segment's fields.
  auto lookup_chunk = [&](uint32_t c, bool in_table) {
    const uint32_t i = c * CHUNK + tid;
    if (tid < CHUNK && i < count) {
      const uint32_t t = t_begin + i;
      uint32_t lo = 0, hi = nseg;
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if ((in_table ? s_t0[mid] : segs[mid].tile0) <= t) lo = mid; else hi = mid;
      }
      const Seg sg = segs[lo];
      TileInfo ti;
      ti.off = sg.off; ti.len = sg.len; ti.pkey = sg.pkey; ti.seg = lo; ti.pval = sg.pval;
      ti.parity = sg.parity | (int32_t)((t - sg.tile0) << 1);   // tile index within segment
      ti.pad = sg.depth;
      s_info[(c & 1) * CHUNK + tid] = ti;
    }
  };

  // Byte range of tile i that is copied in bulk; the array tail that is not a whole
  // 16-byte group is read with plain loads by the issuing thread.
  auto issue = [&](uint32_t i) {
    const int st = i % STAGES;
    // Failure-path test (BQS_OPT_TEST_STALL): the first tile of block 0 is never
    // requested, so its mbarrier phase never completes and the bounded waits run out.
    if (P.test_stall && blockIdx.x == 0 && i == 0) return;
    const TileInfo& ti = s_info[((i / CHUNK) & 1) * CHUNK + (i % CHUNK)];
    const int64_t abase = tile_origin(ti.off) + (int64_t)(ti.parity >> 1) * TILE;
    const int64_t lo = max(abase, ti.off), hi = min(abase + TILE, ti.off + ti.len);
    const int64_t n4 = n_total & ~(int64_t)3;
    const int64_t b0 = lo & ~(int64_t)3;
    const int64_t b1 = min((hi + 3) & ~(int64_t)3, n4);
    const U* src = (const U*)P.b.key[ti.parity & 1];
    const uint32_t* vsrc = P.b.val[ti.parity & 1];
    U* dk = s_in + (size_t)st * TILE;
    uint32_t* dv = s_vin + (size_t)st * TILE;
    for (int64_t j = max(b1, lo); j < hi; ++j) {      // tail keys beyond the last group
      dk[j - abase] = src[j];
      if constexpr (PAIRS) dv[j - abase] = vsrc[j];
    }
    const uint32_t kbytes = b1 > b0 ? (uint32_t)((b1 - b0) * sizeof(U)) : 0u;
    const uint32_t vbytes = (PAIRS && b1 > b0) ? (uint32_t)((b1 - b0) * 4) : 0u;
    mbar_arrive_expect_tx(&s_bar[st], kbytes + vbytes);
    if (kbytes) bulk_g2s(dk + (b0 - abase), src + b0, kbytes, &s_bar[st]);
    if (vbytes) bulk_g2s(dv + (b0 - abase), vsrc + b0, vbytes, &s_bar[st]);
  };

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&s_bar[s], 1);
    s_abort = 0;
    fence_mbar_init();
  }
  if (table) {
    uint32_t* t0 = reinterpret_cast<uint32_t*>(s_out);
    for (uint32_t j = tid; j < nseg; j += THREADS) t0[j] = segs[j].tile0;
    __syncthreads();
  }
  lookup_chunk(0, table);
  if (count > CHUNK) lookup_chunk(1, table);
  __syncthreads();
  if (tid == 0)
    for (uint32_t i = 0; i < (uint32_t)STAGES && i < count; ++i) issue(i);

  uint32_t i = 0;
  bool aborted = false;   // the whole block left the loop after a wait gave up
  for (; i < count; ++i) {
    const int st = i % STAGES;
    const uint32_t parity = (i / STAGES) & 1;
    if (i > 0 && i % CHUNK == 0 && (i / CHUNK + 1) * CHUNK < count) {
      // Entering chunk c = i/CHUNK: chunk c-1 is finished, its slot takes chunk c+1
      // (needed once the refills run STAGES tiles ahead into it).
      lookup_chunk(i / CHUNK + 1, false);
    }
    // Every thread waits for the tile itself (the mbarrier's acquire makes the bulk copy
    // visible to it); a wait that gave up is acted on at the first block barrier below,
    // which every thread reaches, so the whole block leaves the loop together.
    const bool waited = mbar_wait_bounded(&s_bar[st], parity, P.ctrl, P.wait_limit);

    const TileInfo ti = s_info[((i / CHUNK) & 1) * CHUNK + (i % CHUNK)];
    const int64_t abase = tile_origin(ti.off) + (int64_t)(ti.parity >> 1) * TILE;
    const int lo = (int)(max(abase, ti.off) - abase);
    const int hi = (int)(min(abase + TILE, ti.off + ti.len) - abase);
    const bool full = lo == 0 && hi == TILE;
    const CT cp = Cmp<KT>::of((U)ti.pkey);
    const uint32_t pv = ti.pval;
    const U* tk = s_in + (size_t)st * TILE;
    const uint32_t* tv = s_vin + (size_t)st * TILE;

    // Scan phase: keys from shared memory.  Keys outside the segment are replaced by
    // the pivot, so they count as "equal" and are neither counted nor moved.
    U key[KPT];
    uint32_t val[PAIRS ? KPT : 1];
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      union { uint4 v; U e[VEC]; } u;
      u.v = *reinterpret_cast<const uint4*>(tk + (j * THREADS + tid) * VEC);
#pragma unroll
      for (int e = 0; e < VEC; ++e) key[j * VEC + e] = u.e[e];
      if constexpr (PAIRS) {
#pragma unroll
        for (int e = 0; e < VEC; ++e) val[j * VEC + e] = tv[(j * THREADS + tid) * VEC + e];
      }
    }
    if (!full) {
#pragma unroll
      for (int r = 0; r < KPT; ++r) {
        const int idx = ((r / VEC) * THREADS + tid) * VEC + (r % VEC);
        const bool valid = idx >= lo && idx < hi;
        key[r] = valid ? key[r] : (U)ti.pkey;
        if constexpr (PAIRS) val[r] = valid ? val[r] : pv;
      }
    }
    CT kc[KPT];
    uint32_t cl = 0, cg = 0;   // the thread's outcome counts (its share of the buffer)
#pragma unroll
    for (int r = 0; r < KPT; ++r) {
      kc[r] = Cmp<KT>::of(key[r]);
      const uint32_t v = PAIRS ? val[r] : 0u;
      cl += cmp_less<PAIRS>(kc[r], v, cp, pv);
      cg += cmp_less<PAIRS>(cp, pv, kc[r], v);
    }
    // Offsets: exclusive scan of the packed counts over the warp (shuffles), then a
    // prefix over the warp totals.
    const uint32_t own = cl | (cg << 16);
    uint32_t incl = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(~0u, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_wcnt[warp] = incl;
    // This barrier also orders the reuse of s_out, s_wcnt and s_base after the previous
    // tile's write-out (no thread stages before every thread is past that write-out).
    if (__syncthreads_or(!waited)) {
      if (tid == 0) s_abort = 1;
      aborted = true;
      break;
    }
    uint32_t off_lt = 0, off_gt = 0, nlt = 0, ngt = 0;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) {
      const uint32_t c = s_wcnt[w];
      if (w < warp) { off_lt += c & 0xFFFF; off_gt += c >> 16; }
      nlt += c & 0xFFFF;
      ngt += c >> 16;
    }
    // Reservation of both runs: one atomic per tile.  Its result is stored only after
    // the staging below, so the atomic's latency overlaps that work.
    unsigned long long my_base = 0;
    if (tid == 0)
      my_base = atomicAdd(&cursor[ti.seg], (unsigned long long)nlt | ((unsigned long long)ngt << 32));

    // Rearrangement into output order in shared memory: the thread's "<" keys go to
    // consecutive slots from its exclusive prefix, its ">" keys likewise after all "<".
    const uint32_t excl = incl - own;
    uint32_t pl = off_lt + (excl & 0xFFFF), pg = nlt + off_gt + (excl >> 16);
#pragma unroll
    for (int r = 0; r < KPT; ++r) {
      const uint32_t v = PAIRS ? val[r] : 0u;
      const bool l = cmp_less<PAIRS>(kc[r], v, cp, pv);
      const bool g = cmp_less<PAIRS>(cp, pv, kc[r], v);
      if (l) {
        s_out[pl] = key[r];
        if constexpr (PAIRS) s_vout[pl] = val[r];
      }
      if (g) {
        s_out[pg] = key[r];
        if constexpr (PAIRS) s_vout[pg] = val[r];
      }
      pl += l;
      pg += g;
    }
    if (tid == 0) s_base = my_base;
    __syncthreads();   // staging complete, s_base visible, tile buffer st no longer read

    if (tid == 0 && i + STAGES < count) issue(i + STAGES);   // refill this stage

    // Rearrangement: coalesced write-out of the two runs.
    const unsigned long long base = s_base;
    U* dst = (U*)P.b.key[(ti.parity & 1) ^ 1];
    uint32_t* vdst = P.b.val[(ti.parity & 1) ^ 1];
    const int64_t left = ti.off + (int64_t)(uint32_t)base;
    const int64_t right = ti.off + ti.len - (int64_t)(uint32_t)(base >> 32) - ngt;
    U* dl = dst + left;
#pragma unroll 4
    for (uint32_t j = tid; j < nlt; j += THREADS) dl[j] = s_out[j];
    U* dr = dst + right;
    const U* so = s_out + nlt;
#pragma unroll 4
    for (uint32_t j = tid; j < ngt; j += THREADS) dr[j] = so[j];
    if constexpr (PAIRS) {
      uint32_t* vl = vdst + left;
      for (uint32_t j = tid; j < nlt; j += THREADS) vl[j] = s_vout[j];
      uint32_t* vr = vdst + right;
      for (uint32_t j = tid; j < ngt; j += THREADS) vr[j] = s_vout[nlt + j];
    }
    // No barrier here: the next tile's first barrier orders every reuse of s_out, s_wcnt
    // and s_base after this write-out, and the descriptor slot that a lookup at the next
    // tile may refill belongs to a finished chunk.
    if constexpr (FUSED) {
      // Fused bookkeeping (levels of few tiles per block): every finished tile adds its
      // counts to its segment's completion word (thread 0, one acquire-release atomic
      // after a block barrier, which publishes the tile's write-out); the block whose
      // tile completes the segment does the segment's bookkeeping at once with one
      // warp, from the tile's descriptor and the word's totals, and the block that
      // completes the level's last segment copies the control block out and empties the
      // level's consumed lists.
      __syncthreads();
      if (tid == 0) {
        const unsigned long long mine = done_word(nlt, ngt);
        const unsigned long long tot = atomic_add_acq_rel(&P.l.tdone[pp][ti.seg], mine) + mine;
        const uint32_t nt = (uint32_t)tile_count(ti.off, ti.len, TILE);
        s_done_seg = (uint32_t)(tot >> (2 * kDoneShift)) == nt ? ti.seg : ~0u;
        s_done_word = tot;
      }
      __syncthreads();
      if (s_done_seg != ~0u) {
        if (warp == 0) {
          constexpr unsigned long long kField = (1ull << kDoneShift) - 1;
          const unsigned long long tot = s_done_word;
          Seg sg;
          sg.off = ti.off; sg.len = ti.len; sg.pkey = ti.pkey; sg.pval = ti.pval;
          sg.depth = ti.pad; sg.parity = ti.parity & 1; sg.tile0 = 0;
          bookkeep_children<KT, PAIRS>(P, pp, pp ^ 1, lane == 0, sg, (int64_t)(tot & kField),
                                       (int64_t)((tot >> kDoneShift) & kField));
          __syncwarp();
          if (lane == 0) s_copy = atomic_add_acq_rel_u32(&P.ctrl->bk_done, 1u) + 1 == nseg;
        }
        __syncthreads();
        if (s_copy && P.ctrl_host) copy_ctrl_out(P, pp);
      }
    }
  }
  if (s_abort && tid == 0) {
    // Let the copies already issued (tiles i .. i+STAGES-1) land before the block's
    // shared memory goes away; each of these waits is bounded too.
    for (uint32_t j = i; j < count && j < i + STAGES; ++j)
      (void)mbar_wait_bounded(&s_bar[j % STAGES], (j / STAGES) & 1, P.ctrl, P.wait_limit);
  }
  // With fused bookkeeping a block that gave up copies the control block out itself (its
  // status word holds the timeout): the level's last segment may never complete.
  if constexpr (FUSED) {
    if (P.ctrl_host && aborted) copy_ctrl_out(P, -1);
  }
}

}  // namespace bqs

// Bitonic sorting networks (Batcher 1968) held in registers, and the shared-memory
// staging helpers they use.
//
// m = 2^k entries (order images, padded with the largest key) are sorted by a fixed
// network with no data-dependent branches.  Each of T threads holds R consecutive
// entries in registers (entry e = thread * R + i), so
//   * exchanges between entries less than R apart are register compare-exchanges,
//   * exchanges between threads of one warp use __shfl_xor_sync (or, for 32-bit keys
//     with R = 32, register compare-exchanges after a transpose of the warp's block),
//   * only exchanges between warps go through shared memory.
// Used by the small-segment sorts (bqs_small.cuh) and the pivot-sample sort.
#pragma once

#include "bqs_common.cuh"

namespace bqs {

// Barrier of the T threads that run one network together.  A network whose group is
// the whole block (the network kernels) uses the block barrier; with NB several groups
// share one block (the single-block local sort) and each uses its own named barrier,
// 1 + the group's index (barrier 0 is __syncthreads), over T threads.  NB is a
// template flag because a kernel that may name a barrier by a register is given all
// 16 of the block's barriers, which lowers how many of its blocks fit on an SM.  A
// warp needs only __syncwarp.
template <int T, bool NB = false>
__device__ __forceinline__ void sync_group() {
  static_assert(T % 32 == 0, "groups are whole warps");
  if constexpr (T == 32) {
    __syncwarp();
  } else if constexpr (!NB) {
    __syncthreads();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)(threadIdx.x / T)), "n"(T) : "memory");
  }
}

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

constexpr int ilog2_c(int v) { return v <= 1 ? 0 : 1 + ilog2_c(v >> 1); }

// Staging layout for rows of R entries (row t = the entries thread t holds).
//  * Rows of 16 eight-byte entries (128 bytes) are padded by 16 bytes: row r starts at
//    entry r * (R + 2).  16-byte accesses to one chunk of 8 consecutive rows then touch
//    8 different bank groups, a whole row read by consecutive threads (the transposes)
//    is contiguous, and the address of entry (r, c) is plain arithmetic.  (For rows of
//    32 four-byte entries the XOR form below measured slightly faster.)
//  * Other rows are XOR-swizzled: entry e of row e / R lives at pos(e), its 16-byte
//    chunk index within the row XORed with key(row), with the same two properties for
//    16-byte row accesses and striped accesses (entry i*T + t by thread t) by a warp, or
//    a half warp for 8-byte keys.  Rows shorter than one chunk are left as they are.
template <class U, int R>
struct RowSwizzle {
  static constexpr int EPC = 16 / (int)sizeof(U);        // entries per 16-byte chunk
  static constexpr bool kChunked = R >= EPC;
  static constexpr int C = kChunked ? R / EPC : 1;        // chunks per row
  static constexpr int LOGC = ilog2_c(C);
  static constexpr bool kPadded = sizeof(U) == 8 && R * (int)sizeof(U) == 128;
  static constexpr int STRIDE = kPadded ? R + EPC : R;    // entries between row starts
  __device__ static __forceinline__ int key(int row) {
    if constexpr (!kChunked || kPadded) return 0;
    else if constexpr (LOGC >= 3) return row & 7;
    else return (row >> (3 - LOGC)) & (C - 1);
  }
  __device__ static __forceinline__ int pos(int e) {
    if constexpr (kPadded) return e + (e / R) * EPC;
    else return e ^ (key(e / R) * EPC);
  }
};

// Staging entries for T rows of R entries.
template <class U, int R, int T>
constexpr int staging_entries() { return T * RowSwizzle<U, R>::STRIDE; }

template <int R, class U>
__device__ __forceinline__ void swz_store_row(U* base, int row, const U (&x)[R]) {
  using S = RowSwizzle<U, R>;
  if constexpr (S::kChunked) {
    const int kq = S::key(row);
#pragma unroll
    for (int c = 0; c < S::C; ++c) {
      union { uint4 v; U e[S::EPC]; } u;
#pragma unroll
      for (int w = 0; w < S::EPC; ++w) u.e[w] = x[c * S::EPC + w];
      reinterpret_cast<uint4*>(base)[row * (S::STRIDE / S::EPC) + (c ^ kq)] = u.v;
    }
  } else {
    store_row<R>(base + row * R, x);
  }
}

template <int R, class U>
__device__ __forceinline__ void swz_load_row(const U* base, int row, U (&x)[R]) {
  using S = RowSwizzle<U, R>;
  if constexpr (S::kChunked) {
    const int kq = S::key(row);
#pragma unroll
    for (int c = 0; c < S::C; ++c) {
      union { uint4 v; U e[S::EPC]; } u;
      u.v = reinterpret_cast<const uint4*>(base)[row * (S::STRIDE / S::EPC) + (c ^ kq)];
#pragma unroll
      for (int w = 0; w < S::EPC; ++w) x[c * S::EPC + w] = u.e[w];
    }
  } else {
    load_row<R>(base + row * R, x);
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

// One stage of a merge phase: compare-exchange of the entries J apart.  The lower index
// keeps the minimum (every half-merge runs ascending, see net_sort).
template <bool PAIRS, int R, int T, int J, class U>
__device__ __forceinline__ void net_stage(U (&x)[R], uint32_t (&y)[R], int t, U* s_x, uint32_t* s_y) {
  if constexpr (J < R) {
    // Both entries of every pair are in this thread.
#pragma unroll
    for (int i = 0; i < R; ++i)
      if ((i & J) == 0) cx_up<PAIRS>(x[i], y[i], x[i | J], y[i | J]);
  } else if constexpr (J < 32 * R) {
    // Partner entry: same register of lane t ^ (J / R).
    constexpr int d = J / R;
    const bool keep_min = (t & d) == 0;
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const U p = shfl_xor_any(x[i], d);
      const uint32_t pv = PAIRS ? __shfl_xor_sync(~0u, y[i], d) : 0u;
      keep_one<PAIRS>(x[i], y[i], p, pv, keep_min);
    }
  } else {
    // Partner in another warp: exchange rows through shared memory.
    constexpr int d = J / R;
    const bool keep_min = (t & d) == 0;
    swz_store_row<R>(s_x, t, x);
    if constexpr (PAIRS) swz_store_row<R>(s_y, t, y);
    __syncthreads();
    U p[R];
    uint32_t pv[R];
    swz_load_row<R>(s_x, t ^ d, p);
    if constexpr (PAIRS) swz_load_row<R>(s_y, t ^ d, pv);
#pragma unroll
    for (int i = 0; i < R; ++i) keep_one<PAIRS>(x[i], y[i], p[i], PAIRS ? pv[i] : 0u, keep_min);
    __syncthreads();
  }
}

// Stages J, J/2, ..., 1 of one merge phase.
template <bool PAIRS, int R, int T, int J, class U>
__device__ __forceinline__ void net_merge(U (&x)[R], uint32_t (&y)[R], int t, U* s_x, uint32_t* s_y) {
  if constexpr (J > 0) {
    net_stage<PAIRS, R, T, J>(x, y, t, s_x, s_y);
    net_merge<PAIRS, R, T, J / 2>(x, y, t, s_x, s_y);
  }
}

// Merge phases K, 2K, ..., M.  Entering phase K, the entries whose complement state
// changes are flipped: during phase K every entry whose index has bit K set is kept
// complemented (the last phase, K = M, complements nothing).
template <bool PAIRS, int R, int T, int K, class U>
__device__ __forceinline__ void net_phases(U (&x)[R], uint32_t (&y)[R], int t, U* s_x, uint32_t* s_y) {
  constexpr int M = R * T;
  if constexpr (K <= M) {
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int e = t * R + i;
      const bool before = (K >= 4) && ((e & (K >> 1)) != 0);
      const bool now = (K < M) && ((e & K) != 0);
      const U m = (before != now) ? ~U(0) : U(0);
      x[i] ^= m;
      if constexpr (PAIRS) y[i] ^= (uint32_t)m;
    }
    net_merge<PAIRS, R, T, K / 2>(x, y, t, s_x, s_y);
    net_phases<PAIRS, R, T, 2 * K>(x, y, t, s_x, s_y);
  }
}

// Phases K, 2K, ..., R of the network on each thread's own R entries (all stages in
// registers), with the complement states of the full network of R*T entries.
template <int R, int T, int K, class U>
__device__ __forceinline__ void net_phases_upto(U (&x)[R], uint32_t (&y)[R], int t) {
  if constexpr (K <= R) {
    constexpr int M = R * T;
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int e = t * R + i;
      const bool before = (K >= 4) && ((e & (K >> 1)) != 0);
      const bool now = (K < M) && ((e & K) != 0);
      x[i] ^= (before != now) ? ~U(0) : U(0);
    }
    net_merge<false, R, T, K / 2>(x, y, t, (U*)nullptr, (uint32_t*)nullptr);
    net_phases_upto<R, T, 2 * K>(x, y, t);
  }
}

// Sorts the m = R*T entries held as x[R], y[R] by T participating threads (t = thread
// index within the group; entry e = t*R + i), ascending: Batcher's bitonic network.
// Entries are ord images (+ payloads), so bitwise complement reverses their order:
// keeping the entries of every descending half-merge complemented turns it into an
// ascending one, and every compare-exchange becomes a plain min/max.  The phases and
// stages are unrolled by template recursion, so every register index is a constant.
// s_x / s_y: shared scratch of m entries, used only for exchanges between warps.
template <bool PAIRS, int R, int T, class U>
__device__ __forceinline__ void net_sort(U (&x)[R], uint32_t (&y)[R], int t, U* s_x, uint32_t* s_y) {
  net_phases<PAIRS, R, T, 2>(x, y, t, s_x, s_y);
}

// The same network with the phases above R in a loop: each such phase is a short run of
// stages between threads (lane distance d, runtime) followed by the log2(R) register
// stages, whose code is shared by all phases.  The fully unrolled network for R = 32
// is tens of thousands of instructions and stalls on instruction fetch; this form
// keeps one phase body.  Key-only.
template <int R, int T, class U, bool NB = false>
__device__ __forceinline__ void net_sort_looped(U (&x)[R], int t, U* s_x) {
  constexpr int M = R * T;
  uint32_t none[R];   // payload slots of the shared stage code: never read (key-only)
  net_phases_upto<R, T, 2, U>(x, none, t);                         // phases 2 .. R
  for (int k = 2 * R; k <= M; k <<= 1) {
    // Entering phase k: entries of thread t are complemented while bit k of their index
    // (bit k/R of t) is set; before, bit k/2 decided.
    const bool before = (t & (k >> 1) / R) != 0;
    const bool now = k < M && (t & k / R) != 0;
    const U m = before != now ? ~U(0) : U(0);
#pragma unroll
    for (int i = 0; i < R; ++i) x[i] ^= m;
    for (int j = k >> 1; j >= R; j >>= 1) {
      const int d = j / R;
      const bool keep_min = (t & d) == 0;
      if (j < 32 * R) {
#pragma unroll
        for (int i = 0; i < R; ++i) {
          const U p = shfl_xor_any(x[i], d);
          x[i] = keep_min ? umin_(x[i], p) : umax_(x[i], p);
        }
      } else {
        swz_store_row<R>(s_x, t, x);
        sync_group<T, NB>();
        U p[R];
        swz_load_row<R>(s_x, t ^ d, p);
#pragma unroll
        for (int i = 0; i < R; ++i) x[i] = keep_min ? umin_(x[i], p[i]) : umax_(x[i], p[i]);
        sync_group<T, NB>();
      }
    }
    net_merge<false, R, T, R / 2>(x, none, t, s_x, (uint32_t*)nullptr);
  }
}

// 32-bit keys, R = 32: the stages between lanes of one warp (entry bits 5..9) run in
// registers too, after a transpose of the warp's 32 x 32 block (register i of lane l
// <-> register l of lane i) through its shared staging rows.  In the transposed layout
// register i holds entry bits 5..9 = i, so a stage on entry bit 5 + b pairs registers
// i and i ^ 2^b, the lower index keeping the minimum as everywhere else.  A phase with
// two or more such stages pays two transposes (80 shared-memory accesses per thread,
// conflict-free) instead of one shuffle and three ALU operations per key and stage.

// Transposes a warp's 32 x 32 block: afterwards x[i] of lane l is the entry that was
// x[l] of lane i.  wb: the warp's 32 staging rows.
__device__ __forceinline__ void warp_transpose32(uint32_t (&x)[32], int lane, uint32_t* wb) {
  using S = RowSwizzle<uint32_t, 32>;
  swz_store_row<32>(wb, lane, x);                         // row `lane`, 16-byte chunks
  __syncwarp();
#pragma unroll
  for (int i = 0; i < 32; ++i) x[i] = wb[S::pos(i * 32 + lane)];   // column `lane`
  __syncwarp();
}

// Register stages 2^(nb-1), ..., 2, 1 (nb in 1..5) of a transposed block.
__device__ __forceinline__ void transposed_stages(uint32_t (&x)[32], int nb) {
  uint32_t none[32];   // payload slots of the shared stage code: never read (key-only)
  switch (nb) {
    case 5: net_stage<false, 32, 1, 16>(x, none, 0, (uint32_t*)nullptr, (uint32_t*)nullptr);
      [[fallthrough]];
    case 4: net_stage<false, 32, 1, 8>(x, none, 0, (uint32_t*)nullptr, (uint32_t*)nullptr);
      [[fallthrough]];
    case 3: net_stage<false, 32, 1, 4>(x, none, 0, (uint32_t*)nullptr, (uint32_t*)nullptr);
      [[fallthrough]];
    case 2: net_stage<false, 32, 1, 2>(x, none, 0, (uint32_t*)nullptr, (uint32_t*)nullptr);
      [[fallthrough]];
    default: net_stage<false, 32, 1, 1>(x, none, 0, (uint32_t*)nullptr, (uint32_t*)nullptr);
  }
}

template <int T, bool NB = false>
__device__ __forceinline__ void net_sort_transposed(uint32_t (&x)[32], int t, uint32_t* s_x) {
  constexpr int R = 32, M = R * T;
  uint32_t none[R];
  const int lane = t & 31;
  uint32_t* wb = s_x + (t >> 5) * 32 * RowSwizzle<uint32_t, 32>::STRIDE;
  net_phases_upto<R, T, 2, uint32_t>(x, none, t);                  // phases 2 .. 32
  for (int k = 2 * R; k <= M; k <<= 1) {
    const bool before = (t & (k >> 1) / R) != 0;
    const bool now = k < M && (t & k / R) != 0;
    const uint32_t m = before != now ? ~0u : 0u;
#pragma unroll
    for (int i = 0; i < R; ++i) x[i] ^= m;
    int j = k >> 1;
    for (; j >= 32 * R; j >>= 1) {                // between warps: shared-memory rows
      const int d = j / R;
      const bool keep_min = (t & d) == 0;
      swz_store_row<R>(s_x, t, x);
      sync_group<T, NB>();
      uint32_t p[R];
      swz_load_row<R>(s_x, t ^ d, p);
#pragma unroll
      for (int i = 0; i < R; ++i) x[i] = keep_min ? umin_(x[i], p[i]) : umax_(x[i], p[i]);
      sync_group<T, NB>();
    }
    if (j == R) {                                 // one lane stage: a shuffle
      const bool keep_min = (t & 1) == 0;
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const uint32_t p = __shfl_xor_sync(~0u, x[i], 1);
        x[i] = keep_min ? umin_(x[i], p) : umax_(x[i], p);
      }
    } else {                                      // stages j .. R: transposed
      warp_transpose32(x, lane, wb);
      transposed_stages(x, 31 - __clz(j / R) + 1);
      warp_transpose32(x, lane, wb);
    }
    net_merge<false, R, T, R / 2>(x, none, t, s_x, (uint32_t*)nullptr);
  }
}

// ---- the flip form of the network, with padding skipped (32-bit keys, R = 32) -----------
//
// Every merge phase k of Batcher's network can start with a "flip" stage, which pairs
// entry e with e ^ (k - 1) inside its block of k entries, and continue with half-
// cleaners (e with e ^ j, j = k/4 .. 1).  All comparators are then ascending (the lower
// entry keeps the minimum) and, after every phase, every block of k entries is sorted
// ascending.  So padding with the largest key, placed at the top (entries len and up),
// stays where it is through the whole network: every comparator that touches an entry
// at or above len leaves both entries as they are.  A warp whose 32 x 32 entries all lie
// at or above len therefore has nothing to do, and the warps below it never need its
// entries.  Only the first ceil(len / 1024) warps of the group work; they synchronise
// among themselves on named barrier 1.  No entry is ever complemented.

// Barrier of the `act` working warps (named barrier 1; a single warp needs none).
__device__ __forceinline__ void sync_active(int act) {
  if (act == 1) __syncwarp();
  else asm volatile("bar.sync 1, %0;" ::"r"(act * 32) : "memory");
}

// Register half-cleaners J, J/2, ..., 1 (entry bits of the register index).
template <int J>
__device__ __forceinline__ void hc_regs32(uint32_t (&x)[32]) {
  if constexpr (J >= 1) {
#pragma unroll
    for (int i = 0; i < 32; ++i)
      if ((i & J) == 0) {
        const uint32_t lo = umin_(x[i], x[i | J]), hi = umax_(x[i], x[i | J]);
        x[i] = lo;
        x[i | J] = hi;
      }
    hc_regs32<J / 2>(x);
  }
}

// Phases 2 .. 32 on a thread's own 32 entries: flip stage, then half-cleaners.
template <int K>
__device__ __forceinline__ void flip_phases_regs32(uint32_t (&x)[32]) {
  if constexpr (K <= 32) {
#pragma unroll
    for (int i = 0; i < 32; ++i)
      if ((i & (K / 2)) == 0) {
        const int u = i ^ (K - 1);
        const uint32_t lo = umin_(x[i], x[u]), hi = umax_(x[i], x[u]);
        x[i] = lo;
        x[u] = hi;
      }
    hc_regs32<K / 4>(x);
    flip_phases_regs32<K * 2>(x);
  }
}

// Half-cleaners of a transposed block on register bits nb-1 .. 0 (nb in 1..5).
__device__ __forceinline__ void transposed_hc32(uint32_t (&x)[32], int nb) {
  switch (nb) {
    case 5: hc_regs32<16>(x); break;
    case 4: hc_regs32<8>(x); break;
    case 3: hc_regs32<4>(x); break;
    case 2: hc_regs32<2>(x); break;
    default: hc_regs32<1>(x);
  }
}

// Compare-exchange of a thread's 32 entries with the staged row pt of its partner
// thread, 16 bytes at a time (at most four partner entries live): entry i meets the
// partner's entry i, or 31 - i when REV (a flip stage); the lower thread keeps minima.
template <bool REV>
__device__ __forceinline__ void cx_with_row32(uint32_t (&x)[32], const uint32_t* s_x, int pt,
                                              bool lower) {
  using S = RowSwizzle<uint32_t, 32>;
  const int kq = S::key(pt);
#pragma unroll
  for (int c = 0; c < S::C; ++c) {
    const uint4 v = reinterpret_cast<const uint4*>(s_x)[pt * (S::STRIDE / S::EPC) + (c ^ kq)];
    const uint32_t e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int i = REV ? 31 - (c * 4 + w) : c * 4 + w;
      x[i] = lower ? umin_(x[i], e[w]) : umax_(x[i], e[w]);
    }
  }
}

// Sorts M = 32 * T entries (entry e = t * 32 + i in register i of network thread t,
// padded with 0xFFFFFFFF from entry len on) ascending.  Only network threads of the
// first `act` = ceil(len / 1024) warps call it; s_x holds the group's staging rows
// (row t for network thread t), wb the 32 rows of the calling warp.
template <int T>
__device__ __forceinline__ void net_sort_flip32(uint32_t (&x)[32], int t, uint32_t* s_x, int act) {
  constexpr int R = 32, M = R * T;
  const int lane = t & 31;
  uint32_t* wb = s_x + (t >> 5) * 32 * RowSwizzle<uint32_t, 32>::STRIDE;
  // Lane half-cleaners j .. R of a phase (j <= 16 R): a shuffle for one stage, a warp
  // transpose around register stages for more.
  auto lane_hc = [&](int j) {
    if (j == R) {
      const bool lower = (lane & 1) == 0;
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const uint32_t p = __shfl_xor_sync(~0u, x[i], 1);
        x[i] = lower ? umin_(x[i], p) : umax_(x[i], p);
      }
    } else if (j > R) {
      warp_transpose32(x, lane, wb);
      transposed_hc32(x, 31 - __clz(j / R) + 1);
      warp_transpose32(x, lane, wb);
    }
  };
  flip_phases_regs32<2>(x);                                     // phases 2 .. 32
  // Phases 64 .. 1024, inside each warp: the flip pairs lane ^ m, register 31 - i, and
  // the lane whose entries are in the lower half of the block keeps the minimum.
#pragma unroll 1
  for (int k = 2 * R; k <= M && k <= 32 * R; k <<= 1) {
    const int m = k / R - 1;
    const bool lower = (lane & ((m + 1) >> 1)) == 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const uint32_t a = __shfl_xor_sync(~0u, x[31 - i], m);
      const uint32_t b = __shfl_xor_sync(~0u, x[i], m);
      x[i] = lower ? umin_(x[i], a) : umax_(x[i], a);
      x[31 - i] = lower ? umin_(x[31 - i], b) : umax_(x[31 - i], b);
    }
    lane_hc(k >> 2);
    hc_regs32<16>(x);
  }
  // Phases 2048 .. M, across warps: the flip and the half-cleaners between warps go
  // through the staging rows (the flip reads the partner's row backwards).  The rows of
  // warps without data hold padding from the load, so a partner there changes nothing.
#pragma unroll 1
  for (int k = 64 * R; k <= M; k <<= 1) {
    int d = k / R - 1;
    bool rev = true;
#pragma unroll 1
    for (int j = k >> 1; j >= 32 * R; j >>= 1) {
      const int pt = t ^ d;
      const bool lower = (t & (j / R)) == 0;
      swz_store_row<R>(s_x, t, x);
      sync_active(act);
      if ((pt >> 5) < act) {
        if (rev) cx_with_row32<true>(x, s_x, pt, lower);
        else cx_with_row32<false>(x, s_x, pt, lower);
      }
      sync_active(act);
      d = (j >> 1) / R;
      rev = false;
    }
    lane_hc(16 * R);
    hc_regs32<16>(x);
  }
}

// 64-bit keys, R = 16: entry bits 0..3 are register bits and 4..8 lane bits.  Each
// half warp transposes its 16 x 16 block (register i of lane l <-> register l of lane
// i within the half), which brings entry bits 4..7 into the registers; bit 8 (lane
// bit 4) stays a shuffle with the other half warp, bits above a shared-memory
// exchange between warps.  Each half warp's block is 16 padded staging rows.

__device__ __forceinline__ void halfwarp_transpose16(uint64_t (&x)[16], int lane, uint64_t* wb) {
  using S = RowSwizzle<uint64_t, 16>;
  swz_store_row<16>(wb, lane, x);                          // row `lane` of the warp's 32
  __syncwarp();
  const int h = lane & 16, c = lane & 15;
#pragma unroll
  for (int i = 0; i < 16; ++i) x[i] = wb[S::pos((h + i) * 16 + c)];   // column c of the half
  __syncwarp();
}

// Register stages 2^(nb-1), ..., 1 (nb in 1..4) of a transposed 16-entry row.
__device__ __forceinline__ void transposed_stages16(uint64_t (&x)[16], int nb) {
  uint32_t none[16];   // payload slots of the shared stage code: never read (key-only)
  switch (nb) {
    case 4: net_stage<false, 16, 1, 8>(x, none, 0, (uint64_t*)nullptr, (uint32_t*)nullptr);
      [[fallthrough]];
    case 3: net_stage<false, 16, 1, 4>(x, none, 0, (uint64_t*)nullptr, (uint32_t*)nullptr);
      [[fallthrough]];
    case 2: net_stage<false, 16, 1, 2>(x, none, 0, (uint64_t*)nullptr, (uint32_t*)nullptr);
      [[fallthrough]];
    default: net_stage<false, 16, 1, 1>(x, none, 0, (uint64_t*)nullptr, (uint32_t*)nullptr);
  }
}

template <int T, bool NB = false>
__device__ __forceinline__ void net_sort_transposed64(uint64_t (&x)[16], int t, uint64_t* s_x) {
  constexpr int R = 16, M = R * T;
  uint32_t none[R];
  const int lane = t & 31;
  uint64_t* wb = s_x + (t >> 5) * 32 * RowSwizzle<uint64_t, 16>::STRIDE;
  auto lane_stage = [&](int d) {
    const bool keep_min = (t & d) == 0;
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const uint64_t p = __shfl_xor_sync(~0u, (unsigned long long)x[i], d);
      x[i] = keep_min ? umin_(x[i], p) : umax_(x[i], p);
    }
  };
  net_phases_upto<R, T, 2, uint64_t>(x, none, t);                  // phases 2 .. 16
  for (int k = 2 * R; k <= M; k <<= 1) {
    const bool before = (t & (k >> 1) / R) != 0;
    const bool now = k < M && (t & k / R) != 0;
    const uint64_t m = before != now ? ~0ull : 0ull;
#pragma unroll
    for (int i = 0; i < R; ++i) x[i] ^= m;
    int j = k >> 1;
    for (; j >= 32 * R; j >>= 1) {                // between warps: shared-memory rows
      const int d = j / R;
      const bool keep_min = (t & d) == 0;
      swz_store_row<R>(s_x, t, x);
      sync_group<T, NB>();
      uint64_t p[R];
      swz_load_row<R>(s_x, t ^ d, p);
#pragma unroll
      for (int i = 0; i < R; ++i) x[i] = keep_min ? umin_(x[i], p[i]) : umax_(x[i], p[i]);
      sync_group<T, NB>();
    }
    if (j == 16 * R) {                            // entry bit 8: the other half warp
      lane_stage(16);
      j >>= 1;
    }
    if (j == R) {                                 // entry bit 4 alone: a shuffle
      lane_stage(1);
    } else if (j > R) {                           // entry bits 4 .. log2(j): transposed
      halfwarp_transpose16(x, lane, wb);
      transposed_stages16(x, 31 - __clz(j / R) + 1);
      halfwarp_transpose16(x, lane, wb);
    }
    net_merge<false, R, T, R / 2>(x, none, t, s_x, (uint32_t*)nullptr);
  }
}

}  // namespace bqs

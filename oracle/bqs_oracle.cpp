// BlockQuicksort CPU oracle -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.
//
// A plain, slow, single-threaded restatement of BlockQuicksort (Edelkamp & Weiss,
// "BlockQuicksort: How Branch Mispredictions don't affect Quicksort", arXiv 1604.06697).
// It exists only to check the CUDA path: only tests/, __graft_entry__.smoke() and the
// cpu_baseline / reference leg of bench.py may load it.  It shares no code, header,
// table or helper with the CUDA library, and the CUDA library never calls it.
//
// What it computes, part by part (all citations are to the paper):
//   * Quicksort main loop (Sec. 2 "Quicksort and improvements", Algorithm 1, and the
//     main loop of Appendix B): explicit stack, the larger side is stacked and the loop
//     continues on the smaller side; the pivot is excluded from both sides; Introsort
//     depth limit 2*floor(log2 n)+3 with Heapsort for an over-deep sub-array;
//     Insertionsort for sub-arrays of at most 16 elements.
//   * Pivot selection (Sec. 2 and Sec. 4 "Different Pivot Selection Methods"):
//     median-of-three of (first, middle, last), and median of a sqrt(n) sample which
//     falls back to median-of-five-medians-of-five below 20000 elements and to
//     median-of-three for small arrays.
//   * Block partitioning (Sec. 3, Algorithm 3) with B = 128, including the final scan
//     of the at most 2B remaining elements and the compaction of the one buffer that may
//     still hold misplaced elements (Sec. 3, the "basic variant" of Appendix B).
//   * The plain definition of a value partition (Sec. 2 "Quicksort and improvements":
//     smaller-or-equal left, greater-or-equal right), in its stable "count(<pivot)" form.
//
// Readings where the paper is silent or garbled:
//   * Algorithm 3's scanning comparisons are printed with the directions swapped; the
//     prose of Sec. 3 fixes them: the left buffer collects elements >= pivot, the right
//     buffer elements <= pivot.
//   * The median-of-three sample is (first, first + floor(len/2), last).
//   * sqrt(n) sample: k = floor(sqrt(len)) | 1 equally spaced positions
//     b + floor((2i+1) len / (2k)); the pivot is the sample's median (rank (k-1)/2).
//     Median-of-three is used below 64 elements.
//   * float64 is ordered by the total order ord(x) = bits(x) ^ (sign ? ~0 : 1<<63),
//     which equals IEEE "<" on non-NaN values except that -0.0 < +0.0.
//   * Key-value pairs are ordered lexicographically by (key, payload).
//
// Build: g++ -O2 -std=c++17 -shared -fPIC bqs_oracle.cpp -o liboracle_bqs.so

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <utility>
#include <vector>

namespace {

// Block size B: Sec. 3 fixes it at 128 elements for all experiments.
constexpr int64_t kB = 128;

struct Counters {
  uint64_t comparisons = 0;      // every call of the order predicate
  uint64_t partitions = 0;       // calls of the block partitioner from the main loop
  uint64_t insertion_sorts = 0;  // recursion stoppers: Insertionsort
  uint64_t heap_sorts = 0;       // recursion stoppers: Heapsort (depth limit exceeded)
  uint64_t depth_limit = 0;      // the Introsort limit the main loop used
  uint64_t max_depth = 0;        // deepest level at which a partition ran (root = 1)
};

enum PivotRule { kMedianOf3 = 0, kMedianOfSqrt = 1 };

// ---- element types and their strict weak orders ---------------------------------

uint64_t ord_f64(double x) {
  uint64_t u;
  std::memcpy(&u, &x, sizeof u);
  return (u >> 63) ? ~u : (u | (uint64_t(1) << 63));
}

struct LessI32 { bool operator()(int32_t a, int32_t b) const { return a < b; } };
struct LessI64 { bool operator()(int64_t a, int64_t b) const { return a < b; } };
struct LessF64 { bool operator()(double a, double b) const { return ord_f64(a) < ord_f64(b); } };

template <class K>
struct Pair { K key; uint32_t val; };

template <class K, class KeyLess>
struct LessPair {
  bool operator()(const Pair<K>& a, const Pair<K>& b) const {
    KeyLess kl;
    if (kl(a.key, b.key)) return true;
    if (kl(b.key, a.key)) return false;
    return a.val < b.val;
  }
};

int64_t floor_log2(int64_t n) {  // floor(log2 n) for n >= 1, the paper's ilogb(n)
  int64_t r = 0;
  while (n > 1) { n >>= 1; ++r; }
  return r;
}

int64_t isqrt(int64_t n) {
  int64_t r = (int64_t)std::sqrt((double)n);
  while (r * r > n) --r;
  while ((r + 1) * (r + 1) <= n) ++r;
  return r;
}

template <class T, class Less>
struct Sorter {
  Counters& cnt;
  int pivot_rule;
  int64_t is_thresh;     // Insertionsort for sub-arrays of at most this many elements
  int64_t depth_limit;   // < 0: 2*floor(log2 n)+3

  bool lt(const T& a, const T& b) {
    ++cnt.comparisons;
    return Less()(a, b);
  }

  // ---- recursion stoppers ---------------------------------------------------------

  // Insertionsort (textbook, Knuth 5.2.1) on A[b, e).
  void insertion_sort(T* A, int64_t b, int64_t e) {
    ++cnt.insertion_sorts;
    for (int64_t i = b + 1; i < e; ++i) {
      T x = A[i];
      int64_t j = i;
      while (j > b && lt(x, A[j - 1])) {
        A[j] = A[j - 1];
        --j;
      }
      A[j] = x;
    }
  }

  // Heapsort (Williams 1964, with Floyd's bottom-up heap construction) on A[b, e).
  void sift_down(T* H, int64_t root, int64_t n) {
    for (;;) {
      int64_t child = 2 * root + 1;
      if (child >= n) return;
      if (child + 1 < n && lt(H[child], H[child + 1])) ++child;
      if (!lt(H[root], H[child])) return;
      std::swap(H[root], H[child]);
      root = child;
    }
  }
  void heap_sort(T* A, int64_t b, int64_t e) {
    ++cnt.heap_sorts;
    T* H = A + b;
    int64_t n = e - b;
    for (int64_t i = n / 2 - 1; i >= 0; --i) sift_down(H, i, n);
    for (int64_t m = n - 1; m > 0; --m) {
      std::swap(H[0], H[m]);
      sift_down(H, 0, m);
    }
  }

  // ---- pivot selection ------------------------------------------------------------

  // Conditional exchange leaving A[i] <= A[j] (the "sort_pair" step of Appendix B).
  void order2(T* A, int64_t i, int64_t j) {
    if (lt(A[j], A[i])) std::swap(A[i], A[j]);
  }

  // Median of three positions: the three values are put into order in place and the
  // position of the middle one is returned.  Afterwards A[i] <= pivot <= A[k].
  int64_t median_of_3(T* A, int64_t i, int64_t j, int64_t k) {
    order2(A, i, j);
    order2(A, j, k);
    order2(A, i, j);
    return j;
  }

  // Position of the median (rank (m-1)/2) of the values at the positions pos[0, m).
  // The selection step is the library's std::nth_element (the paper does the same).
  int64_t median_position(T* A, std::vector<int64_t> pos) {
    size_t mid = (pos.size() - 1) / 2;
    std::nth_element(pos.begin(), pos.begin() + mid, pos.end(),
                     [&](int64_t x, int64_t y) { return lt(A[x], A[y]); });
    return pos[mid];
  }

  // Equally spaced sample of k positions of A[b, b+len): b + floor((2i+1) len / (2k)).
  static std::vector<int64_t> spaced(int64_t b, int64_t len, int64_t k) {
    std::vector<int64_t> p(k);
    for (int64_t i = 0; i < k; ++i) p[i] = b + ((2 * i + 1) * len) / (2 * k);
    return p;
  }

  // Median of five medians of five (Sec. 4): 25 equally spaced positions in five
  // consecutive groups of five; the median of each group, then the median of those.
  int64_t median_of_5_medians_of_5(T* A, int64_t b, int64_t len) {
    std::vector<int64_t> p = spaced(b, len, 25), medians;
    for (int g = 0; g < 5; ++g)
      medians.push_back(median_position(A, std::vector<int64_t>(p.begin() + 5 * g, p.begin() + 5 * g + 5)));
    return median_position(A, medians);
  }

  // ---- block partitioning (Sec. 3, Algorithm 3) ---------------------------------------

  // What one side of the partition carries from one round to the next: the positions,
  // in the order its last scan met them, of the elements of its last block that belong
  // to the other side and have not been exchanged yet (Sec. 3's offset buffer).
  struct Side {
    int64_t misplaced[kB];
    int64_t head = 0;      // first entry not exchanged yet
    int64_t pending = 0;   // entries not exchanged yet
  };

  // Scan phase (Sec. 3): compares `count` elements with the pivot, walking from `from`
  // upwards (step +1, the left side) or downwards (step -1, the right side), and keeps
  // the positions of the elements that belong to the other side: >= pivot met on the
  // left, <= pivot met on the right.  The position is written every time; only the
  // comparison's outcome decides whether the entry is kept, so the loop body has no
  // branch on the data.
  void scan(const T* A, const T& pivot, int64_t from, int64_t count, int step, Side& s) {
    s.head = 0;
    s.pending = 0;
    for (int64_t i = 0; i < count; ++i) {
      const int64_t at = from + step * i;
      s.misplaced[s.pending] = at;
      s.pending += step > 0 ? !lt(A[at], pivot) : !lt(pivot, A[at]);
    }
  }

  // Rearrangement phase (Sec. 3): exchanges misplaced elements of the two sides in
  // pairs, as many pairs as both sides hold.
  static void exchange(T* A, Side& a, Side& b) {
    const int64_t pairs = std::min(a.pending, b.pending);
    for (int64_t j = 0; j < pairs; ++j) std::swap(A[a.misplaced[a.head + j]], A[b.misplaced[b.head + j]]);
    a.head += pairs;
    a.pending -= pairs;
    b.head += pairs;
    b.pending -= pairs;
  }

  // Partitions A[lo, hi) around the element at position piv.  Returns the pivot's
  // final position p: A[lo, p) <= A[p] <= A(p, hi).
  int64_t block_partition(T* A, int64_t lo, int64_t hi, int64_t piv) {
    // The pivot waits at the last position, outside every scan, until the very end.
    const int64_t home = hi - 1;
    std::swap(A[piv], A[home]);
    const T pivot = A[home];

    // [begin, end) is the part of the array whose elements are not yet known to be on
    // their side.  A side whose last block still holds misplaced elements keeps that
    // block inside the range, at its own edge.
    int64_t begin = lo, end = home;
    Side left, right;
    while (end - begin > 2 * kB) {
      // A side that has nothing left to exchange scans its next block ...
      if (left.pending == 0) scan(A, pivot, begin, kB, +1, left);
      if (right.pending == 0) scan(A, pivot, end - 1, kB, -1, right);
      // ... then misplaced pairs are exchanged, and a block with nothing misplaced
      // left leaves the range.
      exchange(A, left, right);
      if (left.pending == 0) begin += kB;
      if (right.pending == 0) end -= kB;
    }

    // At most 2B elements are left.  A side that still has misplaced elements keeps
    // its block; the other side scans everything else as one shorter block.  When
    // neither has any, the rest is split into two halves, one per side.
    const int64_t rest = end - begin;
    int64_t left_len, right_len;
    if (left.pending) {
      left_len = kB;
      right_len = rest - kB;
      scan(A, pivot, end - 1, right_len, -1, right);
    } else if (right.pending) {
      right_len = kB;
      left_len = rest - kB;
      scan(A, pivot, begin, left_len, +1, left);
    } else {
      left_len = rest / 2;
      right_len = rest - left_len;
      scan(A, pivot, begin, left_len, +1, left);
      scan(A, pivot, end - 1, right_len, -1, right);
    }
    exchange(A, left, right);
    if (left.pending == 0) begin += left_len;
    if (right.pending == 0) end -= right_len;

    // Now at most one side still has misplaced elements, and [begin, end) is exactly
    // the block they are in.  They move to the end of that block that faces the other
    // side, without further comparisons, and the pivot takes the slot between the two
    // sides.  Positions are taken nearest-to-that-end first, so every swap moves a
    // misplaced element past elements that are already on their side.
    if (left.pending) {   // >= pivot, kept in ascending positions: fill from the top
      int64_t slot = end;
      for (int64_t j = left.head + left.pending - 1; j >= left.head; --j)
        std::swap(A[--slot], A[left.misplaced[j]]);
      std::swap(A[home], A[slot]);
      return slot;
    }
    if (right.pending) {  // <= pivot, kept in descending positions: fill from the bottom
      int64_t slot = begin;
      for (int64_t j = right.head + right.pending - 1; j >= right.head; --j)
        std::swap(A[slot++], A[right.misplaced[j]]);
      std::swap(A[home], A[slot]);
      return slot;
    }
    std::swap(A[home], A[begin]);
    return begin;
  }

  // Chooses the pivot of A[b, e) (Sec. 2; Sec. 4 "Different Pivot Selection Methods")
  // and returns its position.  Median-of-three also puts its three sample elements in
  // order, which leaves A[b] <= pivot <= A[e-1]; *ends_done then tells the caller that
  // those two are already on their sides.
  int64_t choose_pivot(T* A, int64_t b, int64_t e, bool* ends_done) {
    const int64_t len = e - b;
    if (pivot_rule == kMedianOf3 || len < 64) {
      *ends_done = true;
      return median_of_3(A, b, b + len / 2, e - 1);
    }
    *ends_done = false;
    if (len < 20000) return median_of_5_medians_of_5(A, b, len);
    return median_position(A, spaced(b, len, isqrt(len) | 1));
  }

  // Chooses a pivot for A[b, e) and partitions; returns the pivot's final position.
  int64_t partition(T* A, int64_t b, int64_t e) {
    ++cnt.partitions;
    bool ends_done = false;
    const int64_t piv = choose_pivot(A, b, e, &ends_done);
    return ends_done ? block_partition(A, b + 1, e - 1, piv) : block_partition(A, b, e, piv);
  }

  // ---- Quicksort main loop --------------------------------------------------------

  void sort(T* A, int64_t n) {
    if (n < 2) return;
    const int64_t limit = depth_limit >= 0 ? depth_limit : 2 * floor_log2(n) + 3;
    cnt.depth_limit = (uint64_t)limit;
    struct Frame { int64_t b, e, depth; };
    std::vector<Frame> stack;
    int64_t b = 0, e = n, depth = 0;
    for (;;) {
      if (depth < limit && e - b > is_thresh) {
        int64_t p = partition(A, b, e);
        ++depth;
        cnt.max_depth = std::max<uint64_t>(cnt.max_depth, (uint64_t)depth);
        // Stack the larger side, continue with the smaller one; p itself is final.
        if (p - b > e - (p + 1)) {
          stack.push_back({b, p, depth});
          b = p + 1;
        } else {
          stack.push_back({p + 1, e, depth});
          e = p;
        }
      } else {
        if (e - b > is_thresh) heap_sort(A, b, e);
        else insertion_sort(A, b, e);
        if (stack.empty()) break;
        b = stack.back().b;
        e = stack.back().e;
        depth = stack.back().depth;
        stack.pop_back();
      }
    }
  }
};

template <class T, class Less>
void run_sort(T* A, int64_t n, int rule, int64_t is_thresh, int64_t depth_limit, Counters& c) {
  Sorter<T, Less> s{c, rule, std::max<int64_t>(is_thresh, 2), depth_limit};
  s.sort(A, n);
}

// The pivot value the sort would choose for A[b, e) of a copy of keys[0, n).
template <class T, class Less>
void run_pivot_value(const T* keys, int64_t n, int rule, int64_t b, int64_t e, T* out) {
  Counters c;
  Sorter<T, Less> s{c, rule, 16, -1};
  std::vector<T> a(keys, keys + n);
  bool ends_done = false;
  *out = a[s.choose_pivot(a.data(), b, e, &ends_done)];
}

template <class T, class Less>
int64_t run_block_partition(T* A, int64_t n, int64_t pivot_pos, Counters& c) {
  Sorter<T, Less> s{c, kMedianOf3, 16, -1};
  return s.block_partition(A, 0, n, pivot_pos);
}

// Plain definition of a value partition: out = (elements < pivot, in input order)
// followed by (elements >= pivot, in input order); returns count(< pivot).
template <class T, class Less>
int64_t run_partition_by_value(const T* keys, int64_t n, T pivot, T* out) {
  Less less;
  int64_t split = 0;
  for (int64_t i = 0; i < n; ++i) split += less(keys[i], pivot);
  int64_t lo = 0, hi = split;
  for (int64_t i = 0; i < n; ++i) {
    if (less(keys[i], pivot)) out[lo++] = keys[i];
    else out[hi++] = keys[i];
  }
  return split;
}

template <class K, class KeyLess>
void run_sort_pairs(K* keys, uint32_t* vals, int64_t n, int rule, Counters& c) {
  std::vector<Pair<K>> a(n);
  for (int64_t i = 0; i < n; ++i) a[i] = Pair<K>{keys[i], vals[i]};
  run_sort<Pair<K>, LessPair<K, KeyLess>>(a.data(), n, rule, 16, -1, c);
  for (int64_t i = 0; i < n; ++i) { keys[i] = a[i].key; vals[i] = a[i].val; }
}

void export_counters(const Counters& c, uint64_t* out) {
  if (!out) return;
  out[0] = c.comparisons;
  out[1] = c.partitions;
  out[2] = c.insertion_sorts;
  out[3] = c.heap_sorts;
  out[4] = c.depth_limit;
  out[5] = c.max_depth;
}

}  // namespace

extern "C" {

// dtype: 0 = int32, 1 = int64, 2 = float64.  pivot_rule: 0 = median-of-3, 1 = sqrt(n).
// counters (optional, 6 x uint64): comparisons, partitions, insertion sorts, heap sorts,
// the depth limit used, the deepest partition level reached.
int oracle_sort(void* keys, int64_t n, int32_t dtype, int32_t pivot_rule, int64_t is_thresh,
                int64_t depth_limit, uint64_t* counters) {
  if (n < 0 || (n > 0 && !keys) || pivot_rule < 0 || pivot_rule > 1) return -1;
  Counters c;
  switch (dtype) {
    case 0: run_sort<int32_t, LessI32>((int32_t*)keys, n, pivot_rule, is_thresh, depth_limit, c); break;
    case 1: run_sort<int64_t, LessI64>((int64_t*)keys, n, pivot_rule, is_thresh, depth_limit, c); break;
    case 2: run_sort<double, LessF64>((double*)keys, n, pivot_rule, is_thresh, depth_limit, c); break;
    default: return -1;
  }
  export_counters(c, counters);
  return 0;
}

// Key-value sort, ordered by (key, payload).  Keys of the given dtype, uint32 payloads.
int oracle_sort_pairs(void* keys, uint32_t* vals, int64_t n, int32_t dtype, int32_t pivot_rule,
                      uint64_t* counters) {
  if (n < 0 || (n > 0 && (!keys || !vals)) || pivot_rule < 0 || pivot_rule > 1) return -1;
  Counters c;
  switch (dtype) {
    case 0: run_sort_pairs<int32_t, LessI32>((int32_t*)keys, vals, n, pivot_rule, c); break;
    case 1: run_sort_pairs<int64_t, LessI64>((int64_t*)keys, vals, n, pivot_rule, c); break;
    case 2: run_sort_pairs<double, LessF64>((double*)keys, vals, n, pivot_rule, c); break;
    default: return -1;
  }
  export_counters(c, counters);
  return 0;
}

// Sorts every segment [seg_offsets[i], seg_offsets[i+1]) on its own.
int oracle_sort_segmented(void* keys, const int64_t* seg_offsets, int64_t nseg, int32_t dtype,
                          int32_t pivot_rule) {
  if (nseg < 0 || (nseg > 0 && !seg_offsets)) return -1;
  for (int64_t s = 0; s < nseg; ++s)
    if (seg_offsets[s + 1] < seg_offsets[s] || seg_offsets[s] < 0) return -1;
  const int64_t size = dtype == 0 ? 4 : 8;
  for (int64_t s = 0; s < nseg; ++s) {
    int rc = oracle_sort((char*)keys + seg_offsets[s] * size, seg_offsets[s + 1] - seg_offsets[s],
                         dtype, pivot_rule, 16, -1, nullptr);
    if (rc) return rc;
  }
  return 0;
}

// Algorithm 3 on the whole array keys[0, n) around the element at pivot_pos.
// Returns the pivot's final position, or -1 on invalid arguments.
int64_t oracle_block_partition(void* keys, int64_t n, int32_t dtype, int64_t pivot_pos,
                               uint64_t* counters) {
  if (n < 1 || !keys || pivot_pos < 0 || pivot_pos >= n) return -1;
  Counters c;
  int64_t p;
  switch (dtype) {
    case 0: p = run_block_partition<int32_t, LessI32>((int32_t*)keys, n, pivot_pos, c); break;
    case 1: p = run_block_partition<int64_t, LessI64>((int64_t*)keys, n, pivot_pos, c); break;
    case 2: p = run_block_partition<double, LessF64>((double*)keys, n, pivot_pos, c); break;
    default: return -1;
  }
  export_counters(c, counters);
  return p;
}

// The pivot the sort chooses for the sub-array keys[b, e) (e - b >= 3) under a pivot
// rule (0 = median-of-3, 1 = sqrt(n)), written to *out; keys are not changed.  A test
// entry: it exposes the pivot rules of Sec. 2 and Sec. 4 to their pins.
int oracle_pivot_value(const void* keys, int64_t n, int32_t dtype, int32_t pivot_rule, int64_t b,
                       int64_t e, void* out) {
  if (!keys || !out || b < 0 || e > n || e - b < 3 || pivot_rule < 0 || pivot_rule > 1) return -1;
  switch (dtype) {
    case 0: run_pivot_value<int32_t, LessI32>((const int32_t*)keys, n, pivot_rule, b, e, (int32_t*)out); return 0;
    case 1: run_pivot_value<int64_t, LessI64>((const int64_t*)keys, n, pivot_rule, b, e, (int64_t*)out); return 0;
    case 2: run_pivot_value<double, LessF64>((const double*)keys, n, pivot_rule, b, e, (double*)out); return 0;
    default: return -1;
  }
}

// The key that a sorted copy of keys[0, n) holds at position k (the k-th order statistic,
// which is the definition of that output position), written to *out.  Used to check
// sampled positions of sorts too large for oracle_sort.  The selection step is the
// library's std::nth_element on a copy, with the same total order as the sort.
int oracle_select(const void* keys, int64_t n, int32_t dtype, int64_t k, void* out) {
  if (n < 1 || !keys || !out || k < 0 || k >= n) return -1;
  switch (dtype) {
    case 0: {
      std::vector<int32_t> a((const int32_t*)keys, (const int32_t*)keys + n);
      std::nth_element(a.begin(), a.begin() + k, a.end(), LessI32());
      *(int32_t*)out = a[k];
      return 0;
    }
    case 1: {
      std::vector<int64_t> a((const int64_t*)keys, (const int64_t*)keys + n);
      std::nth_element(a.begin(), a.begin() + k, a.end(), LessI64());
      *(int64_t*)out = a[k];
      return 0;
    }
    case 2: {
      std::vector<double> a((const double*)keys, (const double*)keys + n);
      std::nth_element(a.begin(), a.begin() + k, a.end(), LessF64());
      *(double*)out = a[k];
      return 0;
    }
    default: return -1;
  }
}

// Plain stable value partition (the definition behind bqs_partition).  pivot points to
// one key of the given dtype.  Returns count(< pivot), or -1 on invalid arguments.
int64_t oracle_partition_by_value(const void* keys, int64_t n, int32_t dtype, const void* pivot,
                                  void* out) {
  if (n < 0 || (n > 0 && (!keys || !out)) || !pivot) return -1;
  switch (dtype) {
    case 0: return run_partition_by_value<int32_t, LessI32>((const int32_t*)keys, n, *(const int32_t*)pivot, (int32_t*)out);
    case 1: return run_partition_by_value<int64_t, LessI64>((const int64_t*)keys, n, *(const int64_t*)pivot, (int64_t*)out);
    case 2: return run_partition_by_value<double, LessF64>((const double*)keys, n, *(const double*)pivot, (double*)out);
    default: return -1;
  }
}

// Keys of the wide element types of Sec. 4 ("Different Element Types"): kind 0 = the
// int32 field at byte `offset` of each record (Record: compared by its first field);
// kind 1 = the squared Euclidean norm of the `count` doubles at `offset` (Vector:
// compared by its norm), summed in component order, each product and sum rounded on
// its own (the library is compiled without contraction into fused multiply-adds).
// Sorting the records is then sorting the (key, record index) pairs -- ties broken by
// the index -- and moving every record to its place.
int oracle_record_keys(const void* records, int64_t n, int32_t record_bytes, int32_t kind,
                       int32_t offset, int32_t count, void* keys) {
  if (n < 0 || !records || !keys || record_bytes <= 0) return -1;
  const unsigned char* rec = static_cast<const unsigned char*>(records);
  for (int64_t i = 0; i < n; ++i) {
    const unsigned char* r = rec + i * record_bytes + offset;
    if (kind == 0) {
      int32_t v;
      std::memcpy(&v, r, 4);
      static_cast<int32_t*>(keys)[i] = v;
    } else if (kind == 1) {
      double s = 0.0;
      for (int32_t c = 0; c < count; ++c) {
        double x;
        std::memcpy(&x, r + 8 * c, 8);
        const double sq = x * x;
        s = s + sq;
      }
      static_cast<double*>(keys)[i] = s;
    } else {
      return -1;
    }
  }
  return 0;
}

}  // extern "C"

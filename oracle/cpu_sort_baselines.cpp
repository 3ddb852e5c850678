// CPU comparison sorts timed beside the GPU sort: the C++ standard library's
// introsort (std::sort, the paper's comparison baseline in Sec. 4) on one thread,
// and the GNU parallel mode's multiway mergesort (__gnu_parallel::sort) on all host
// cores when the compiler offers OpenMP.
//
// MEASUREMENT INFRASTRUCTURE, NOT PART OF THE PRODUCT: only the benchmark's CPU
// baseline leg and the tests load this library.  It shares no code with the CUDA
// path or with the oracle (bqs_oracle.cpp).
//
// Keys are sorted under the same total order as everywhere else: int32/int64 by
// value, float64 by the order image bits ^ (sign ? ~0 : 1<<63), which is IEEE "<"
// except that -0.0 sorts before +0.0 (NaN excluded).
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#include <parallel/algorithm>
#endif

namespace {

inline uint64_t f64_image(double d) {
  uint64_t b;
  std::memcpy(&b, &d, 8);
  return (b >> 63) ? ~b : (b | (1ull << 63));
}

struct F64Less {
  bool operator()(double a, double b) const { return f64_image(a) < f64_image(b); }
};

// Portable parallel fallback: sort `threads` chunks with std::sort, then merge
// neighbouring runs pairwise (each round's merges run concurrently).
template <class T, class Less>
void chunk_sort_merge(T* a, int64_t n, int threads, Less less) {
  if (threads < 2 || n < 4096) {
    std::sort(a, a + n, less);
    return;
  }
  std::vector<int64_t> cut(threads + 1);
  for (int i = 0; i <= threads; ++i) cut[i] = n * i / threads;
  {
    std::vector<std::thread> pool;
    for (int i = 0; i < threads; ++i)
      pool.emplace_back([=] { std::sort(a + cut[i], a + cut[i + 1], less); });
    for (auto& t : pool) t.join();
  }
  std::vector<T> tmp(n);
  T* src = a;
  T* dst = tmp.data();
  for (size_t width = 1; width < (size_t)threads; width *= 2) {
    std::vector<std::thread> pool;
    for (size_t i = 0; i < (size_t)threads; i += 2 * width) {
      const int64_t lo = cut[i];
      const int64_t mid = cut[std::min(i + width, (size_t)threads)];
      const int64_t hi = cut[std::min(i + 2 * width, (size_t)threads)];
      pool.emplace_back([=] { std::merge(src + lo, src + mid, src + mid, src + hi, dst + lo, less); });
    }
    for (auto& t : pool) t.join();
    std::swap(src, dst);
  }
  if (src != a) std::memcpy(a, src, sizeof(T) * n);
}

template <class T, class Less>
int sort_typed(void* keys, int64_t n, int threads, Less less) {
  T* a = static_cast<T*>(keys);
  if (threads <= 1) {
    std::sort(a, a + n, less);
    return 1;
  }
#ifdef _OPENMP
  omp_set_num_threads(threads);
  __gnu_parallel::sort(a, a + n, less);
  return 2;
#else
  chunk_sort_merge(a, n, threads, less);
  return 3;
#endif
}

}  // namespace

extern "C" {

// Sorts n keys in place on `threads` host threads (1: std::sort).  dtype 0 int32,
// 1 int64, 2 float64.  Returns 1 for std::sort, 2 for __gnu_parallel::sort, 3 for
// the chunk-sort-and-merge fallback, -1 for a bad dtype.
int cpu_sort_keys(void* keys, int64_t n, int32_t dtype, int32_t threads) {
  switch (dtype) {
    case 0: return sort_typed<int32_t>(keys, n, threads, std::less<int32_t>());
    case 1: return sort_typed<int64_t>(keys, n, threads, std::less<int64_t>());
    case 2: return sort_typed<double>(keys, n, threads, F64Less());
    default: return -1;
  }
}

// 1 when the library was built with OpenMP (parallel sorts use __gnu_parallel::sort).
int cpu_sort_has_openmp() {
#ifdef _OPENMP
  return 1;
#else
  return 0;
#endif
}

}  // extern "C"

// Sorting wide elements (bqs_sort_records): the paper's Record and Vector element types
// (Sec. 4, "Different Element Types": a Record of 21 ints compared by its first field,
// a Vector of 10 doubles compared by its norm).  Moving whole records through every
// partition level would multiply the traffic by the record size, so the sort is
// indirect: one kernel extracts each record's key and pairs it with the record's index,
// the key-value sort orders the (key, index) pairs -- by key, ties by index, so the
// order is unique and equal keys keep their input order -- and one kernel moves every
// record once to its sorted place.
#include <cstdint>

#include <cuda_runtime.h>

#include "bqs.h"
#include "bqs_common.cuh"
#include "bqs_internal.h"

namespace bqs {
namespace {

// Key of record i: its int32 field at `offset`, or the squared Euclidean norm of the
// `count` doubles starting at `offset`, summed in component order with every product
// and sum rounded to double (no fused multiply-add), so any implementation that follows
// the same order gets the same bits.
__global__ void k_record_keys(const unsigned char* __restrict__ rec, int64_t n, int32_t rb,
                              int32_t kind, int32_t offset, int32_t count, void* keys,
                              uint32_t* __restrict__ idx) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const unsigned char* r = rec + i * rb + offset;
    if (kind == BQS_KEY_I32_FIELD) {
      static_cast<int32_t*>(keys)[i] = *reinterpret_cast<const int32_t*>(r);
    } else {
      const double* v = reinterpret_cast<const double*>(r);
      double s = 0.0;
      for (int c = 0; c < count; ++c) s = __dadd_rn(s, __dmul_rn(v[c], v[c]));
      static_cast<double*>(keys)[i] = s;
    }
    idx[i] = (uint32_t)i;
  }
}

// out[i] = rec[idx[i]], one warp per record: lanes move 4-byte words (records are
// 4-byte multiples and 4-byte aligned).
__global__ void k_gather_records(const unsigned char* __restrict__ rec, int64_t n, int32_t rb,
                                 const uint32_t* __restrict__ idx, unsigned char* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int words = rb >> 2;
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
    const uint32_t* s = reinterpret_cast<const uint32_t*>(rec + (int64_t)idx[i] * rb);
    uint32_t* d = reinterpret_cast<uint32_t*>(out + i * rb);
    for (int w = lane; w < words; w += 32) d[w] = s[w];
  }
}

int grid_for(int64_t items, int per_block) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t g = (items + per_block - 1) / per_block;
  return (int)(g < 8 * (int64_t)sms ? (g > 0 ? g : 1) : 8 * (int64_t)sms);
}

}  // namespace
}  // namespace bqs

using namespace bqs;

extern "C" int bqs_sort_records(void* records, int64_t n, int32_t record_bytes, int32_t key_kind,
                                int32_t key_offset, int32_t key_count, bqs_stream_t stream) {
  clear_stats();
  if (n < 0 || n > (int64_t)0xFFFFFFFFll || record_bytes <= 0 || record_bytes % 4 != 0 ||
      key_offset < 0)
    return BQS_ERR_INVALID;
  if (key_kind == BQS_KEY_I32_FIELD) {
    if (key_offset % 4 != 0 || key_offset + 4 > record_bytes) return BQS_ERR_INVALID;
  } else if (key_kind == BQS_KEY_F64_SQNORM) {
    if (key_count < 1 || record_bytes % 8 != 0 || key_offset % 8 != 0 ||
        (int64_t)key_offset + 8 * (int64_t)key_count > record_bytes)
      return BQS_ERR_INVALID;
  } else {
    return BQS_ERR_INVALID;
  }
  if (n <= 1) return BQS_OK;
  if (!records || ((uintptr_t)records & (key_kind == BQS_KEY_F64_SQNORM ? 7u : 3u)) != 0)
    return BQS_ERR_INVALID;

  const cudaStream_t s = (cudaStream_t)stream;
  const size_t key_bytes = key_kind == BQS_KEY_I32_FIELD ? 4 : 8;
  // keys, then indices, then the gathered records; each part 256-byte aligned
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t o_idx = up((size_t)n * key_bytes);
  const size_t o_out = o_idx + up((size_t)n * 4);
  const size_t total = o_out + (size_t)n * (size_t)record_bytes;
  void* base = nullptr;
  cudaError_t e = cudaMallocAsync(&base, total, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? BQS_ERR_NOMEM : fail_cuda(e, "cudaMallocAsync");
  }
  unsigned char* w = static_cast<unsigned char*>(base);
  void* keys = w;
  uint32_t* idx = reinterpret_cast<uint32_t*>(w + o_idx);
  unsigned char* out = w + o_out;

  int rc = BQS_OK;
  k_record_keys<<<grid_for(n, 256), 256, 0, s>>>(static_cast<const unsigned char*>(records), n,
                                                  record_bytes, key_kind, key_offset, key_count,
                                                  keys, idx);
  e = cudaGetLastError();
  if (e != cudaSuccess) rc = fail_cuda(e, "k_record_keys");
  if (rc == BQS_OK) {
    Call c;
    c.keys = keys;
    c.vals = idx;
    c.n = n;
    c.stream = stream;
    c.opt = current_options();
    rc = dispatch_call(key_kind == BQS_KEY_I32_FIELD ? BQS_INT32 : BQS_FLOAT64, c);
  }
  if (rc == BQS_OK) {
    k_gather_records<<<grid_for(n, 8), 256, 0, s>>>(static_cast<const unsigned char*>(records), n,
                                                    record_bytes, idx, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) rc = fail_cuda(e, "k_gather_records");
  }
  if (rc == BQS_OK) {
    e = cudaMemcpyAsync(records, out, (size_t)n * (size_t)record_bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) rc = fail_cuda(e, "cudaMemcpyAsync(records)");
  }
  e = cudaFreeAsync(base, s);
  if (e != cudaSuccess && rc == BQS_OK) rc = fail_cuda(e, "cudaFreeAsync");
  return rc;
}

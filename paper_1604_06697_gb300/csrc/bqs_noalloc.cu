// Allocation-free sort entry point (bqs_sort_noalloc).
//
// Some callers cannot allocate device memory at the moment they sort: a service that
// reserves all of its GPU memory at start-up and must never grow it or risk an
// out-of-memory failure in the middle of a request, or code embedded in a host
// framework whose own allocator owns the device memory.  This entry point sorts with
// scratch that already exists: a fixed array in the library's device data, sized for
// up to kNoAllocMaxKeys keys.  Every GPU on which the library is loaded holds this
// array until the process exits.
//
// It runs the same kernels as bqs_sort; only the source of the scratch differs.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "bqs.h"
#include "bqs_internal.h"

namespace bqs {
namespace {

constexpr int64_t kNoAllocMaxKeys = int64_t(1) << 20;   // largest n accepted
constexpr size_t kNoAllocBytes = size_t(16) << 20;     // 16 MiB of scratch per device

// The scratch itself.  In host code this name is only a stand-in for the device
// symbol, never a usable address: the device address is looked up per device below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per device.
int scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_cuda(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return kErrUnsupported;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return fail_cuda(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return kOk;
}

}  // namespace
}  // namespace bqs

using namespace bqs;

extern "C" int bqs_sort_noalloc(void* keys, int64_t n, int32_t dtype, bqs_stream_t stream) {
  if (dtype < BQS_INT32 || dtype > BQS_FLOAT64 || n < 0) return BQS_ERR_INVALID;
  if (n > kNoAllocMaxKeys) return BQS_ERR_TOO_LARGE;
  clear_stats();
  // The level loop reads counts back from the device between levels, which a stream
  // that is being captured into a CUDA graph cannot do; such a call is refused before
  // anything is enqueued, so the caller's capture stays valid.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  const cudaError_t ce = cudaStreamIsCapturing((cudaStream_t)stream, &cap);
  if (ce != cudaSuccess) return fail_cuda(ce, "cudaStreamIsCapturing");
  if (cap != cudaStreamCaptureStatusNone) return BQS_ERR_UNSUPPORTED;
  if (n <= 1) return BQS_OK;
  if (!keys || ((uintptr_t)keys & 15u)) return BQS_ERR_INVALID;
  void* ws = nullptr;
  int rc = scratch_address(&ws);
  if (rc) return rc;
  Call c;
  c.keys = keys;
  c.n = n;
  c.stream = stream;
  c.opt = current_options();
  c.fixed_ws = ws;
  c.fixed_ws_bytes = (int64_t)kNoAllocBytes;
  // A layout that needs more than the array (very small cutoffs set through
  // bqs_set_option) is refused before any work is queued.
  if (layout_bytes(n, dtype == BQS_INT32 ? 4 : 8, false, 0, (int)c.opt.small_cutoff) >
      (int64_t)kNoAllocBytes)
    return BQS_ERR_TOO_LARGE;
  // The driver clears every counter and list header it relies on at the start of the
  // call, so what an earlier call left in the shared array does not matter.
  return dispatch_call(dtype, c);
}

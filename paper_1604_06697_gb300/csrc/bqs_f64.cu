// float64 instantiation of the BlockQuicksort driver and kernels.
#include "bqs_driver.cuh"

namespace bqs {
BQS_INSTANTIATE(KeyF64, run_f64)
}  // namespace bqs

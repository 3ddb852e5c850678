// int64 instantiation of the BlockQuicksort driver and kernels.
#include "bqs_driver.cuh"

namespace bqs {
BQS_INSTANTIATE(KeyI64, run_i64)
}  // namespace bqs

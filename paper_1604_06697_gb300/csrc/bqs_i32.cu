// int32 instantiation of the BlockQuicksort driver and kernels.
#include "bqs_driver.cuh"

namespace bqs {
BQS_INSTANTIATE(KeyI32, run_i32)
}  // namespace bqs

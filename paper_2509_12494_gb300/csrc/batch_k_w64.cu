// batch_k_w64.cu -- the persistent kernel for batches of 64-bit transforms only.
#include "batch_kernel.cuh"

namespace mq {
namespace batch_detail {
MQ_DEFINE_PERSISTENT(1, false)
}  // namespace batch_detail
}  // namespace mq

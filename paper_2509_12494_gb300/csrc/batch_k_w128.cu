// batch_k_w128.cu -- the persistent kernel for batches of 128-bit transforms only.
#include "batch_kernel.cuh"

namespace mq {
namespace batch_detail {
MQ_DEFINE_PERSISTENT(2, false)
}  // namespace batch_detail
}  // namespace mq

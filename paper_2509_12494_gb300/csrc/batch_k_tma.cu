// batch_k_tma.cu -- the persistent kernel for batches of 128-bit transforms whose every pass takes
// the TMA form (the prefetching form then carries only that code path).
#include "batch_kernel.cuh"

namespace mq {
namespace batch_detail {
MQ_DEFINE_PERSISTENT(6, false)
}  // namespace batch_detail
}  // namespace mq

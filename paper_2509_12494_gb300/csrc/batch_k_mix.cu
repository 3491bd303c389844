// batch_k_mix.cu -- the persistent kernel for batches of any mix of widths, transforms and BLAS.
#include "batch_kernel.cuh"

namespace mq {
namespace batch_detail {
MQ_DEFINE_PERSISTENT(3, true)
}  // namespace batch_detail
}  // namespace mq

// ntt_w128_inv.cu -- instantiates the inverse transform kernels for 128-bit residues.
#include "ntt_kernel.cuh"

namespace mq {
cudaError_t launch_ntt_w2_inv(int L, const PassArgs &a, cudaStream_t s) {
    return ntt_detail::launch_w<2, true>(L, a, s);
}
}  // namespace mq

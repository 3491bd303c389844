// ntt_w64_inv.cu -- instantiates the inverse transform kernels for 64-bit residues.
#include "ntt_kernel.cuh"

namespace mq {
cudaError_t launch_ntt_w1_inv(int L, const PassArgs &a, cudaStream_t s) {
    return ntt_detail::launch_w<1, true>(L, a, s);
}
}  // namespace mq

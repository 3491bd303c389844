// ntt_w64_fwd.cu -- instantiates the forward transform kernels for 64-bit residues.
#include "ntt_kernel.cuh"

namespace mq {
cudaError_t launch_ntt_w1_fwd(int L, const PassArgs &a, cudaStream_t s) {
    return ntt_detail::launch_w<1, false>(L, a, s);
}
}  // namespace mq

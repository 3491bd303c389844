// ntt_w128_fwd.cu -- instantiates the forward transform kernels for 128-bit residues.
#include "ntt_kernel.cuh"

namespace mq {
cudaError_t launch_ntt_w2_fwd(int L, const PassArgs &a, cudaStream_t s) {
    return ntt_detail::launch_w<2, false>(L, a, s);
}
}  // namespace mq

// polymul_w64.cu -- instantiates the fused polynomial-product kernels for 64-bit residues.
#include "polymul.cuh"

namespace mq {
cudaError_t launch_polymul_w1(int L, const PassArgs &fa, const PassArgs &fb, const PassArgs &ia, const MulArgs &m,
                              cudaStream_t s) {
    return polymul_detail::launch_polymul_w<1>(L, fa, fb, ia, m, s);
}
}  // namespace mq

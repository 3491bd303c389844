// polymul_w128.cu -- instantiates the fused polynomial-product kernels for 128-bit residues.
#include "polymul.cuh"

namespace mq {
cudaError_t launch_polymul_w1(int L, const PassArgs &fa, const PassArgs &fb, const PassArgs &ia, const MulArgs &m,
                              cudaStream_t s);

cudaError_t launch_polymul_w2(int L, const PassArgs &fa, const PassArgs &fb, const PassArgs &ia, const MulArgs &m,
                              cudaStream_t s) {
    return polymul_detail::launch_polymul_w<2>(L, fa, fb, ia, m, s);
}

cudaError_t launch_polymul(int width, int L, const PassArgs &fa, const PassArgs &fb, const PassArgs &ia,
                           const MulArgs &m, cudaStream_t s) {
    return width == 1 ? launch_polymul_w1(L, fa, fb, ia, m, s) : launch_polymul_w2(L, fa, fb, ia, m, s);
}
}  // namespace mq

// ntt_w256_fwd.cu -- instantiates the forward transform kernels for 256-bit residues (tiles up to 2^10).
#include "ntt_kernel.cuh"

namespace mq {
cudaError_t launch_ntt_w4_fwd(int L, const PassArgs &a, cudaStream_t s) {
    switch (L) {
    case 1: return ntt_detail::launch_one<4, 1, false>(a, s);
    case 2: return ntt_detail::launch_one<4, 2, false>(a, s);
    case 3: return ntt_detail::launch_one<4, 3, false>(a, s);
    case 4: return ntt_detail::launch_one<4, 4, false>(a, s);
    case 5: return ntt_detail::launch_one<4, 5, false>(a, s);
    case 6: return ntt_detail::launch_one<4, 6, false>(a, s);
    case 7: return ntt_detail::launch_one<4, 7, false>(a, s);
    case 8: return ntt_detail::launch_one<4, 8, false>(a, s);
    case 9: return ntt_detail::launch_one<4, 9, false>(a, s);
    case 10: return ntt_detail::launch_one<4, 10, false>(a, s);
    default: return cudaErrorInvalidValue;
    }
}
}  // namespace mq

// ntt_w192_inv.cu -- instantiates the inverse transform kernels for 192-bit residues (tiles up to 2^10).
#include "ntt_kernel.cuh"

namespace mq {
cudaError_t launch_ntt_w3_inv(int L, const PassArgs &a, cudaStream_t s) {
    switch (L) {
    case 1: return ntt_detail::launch_one<3, 1, true>(a, s);
    case 2: return ntt_detail::launch_one<3, 2, true>(a, s);
    case 3: return ntt_detail::launch_one<3, 3, true>(a, s);
    case 4: return ntt_detail::launch_one<3, 4, true>(a, s);
    case 5: return ntt_detail::launch_one<3, 5, true>(a, s);
    case 6: return ntt_detail::launch_one<3, 6, true>(a, s);
    case 7: return ntt_detail::launch_one<3, 7, true>(a, s);
    case 8: return ntt_detail::launch_one<3, 8, true>(a, s);
    case 9: return ntt_detail::launch_one<3, 9, true>(a, s);
    case 10: return ntt_detail::launch_one<3, 10, true>(a, s);
    default: return cudaErrorInvalidValue;
    }
}
}  // namespace mq

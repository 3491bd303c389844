// blas_ops.cuh -- the element operation of each modular BLAS kernel (shared by the standalone
// BLAS kernels and the batched persistent kernel).
#pragma once
#include "common.cuh"

namespace mq {

template <int OP>
__device__ __forceinline__ uint4 op128(uint4 a, uint4 b, const Mod128 &m, uint4 s, uint4 sp) {
    if (OP == OP_VADD) return add_mod(a, b, m.q);
    if (OP == OP_VSUB) return sub_mod(a, b, m.q);
    if (OP == OP_VMUL) return mul_mod_barrett(a, b, m);
    return add_mod(mul_mod_shoup(a, s, sp, m.q), b, m.q);  // axpy: s*x + y with x = a, y = b
}

template <int OP>
__device__ __forceinline__ uint64_t op64(uint64_t a, uint64_t b, const Mod64 &m, uint64_t s, uint64_t sp) {
    if (OP == OP_VADD) return add_mod(a, b, m.q);
    if (OP == OP_VSUB) return sub_mod(a, b, m.q);
    if (OP == OP_VMUL) return mul_mod_barrett(a, b, m);
    return add_mod(mul_mod_shoup(a, s, sp, m.q), b, m.q);
}

}  // namespace mq

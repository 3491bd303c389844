// blas_wide.cu -- the element-wise modular BLAS of blas.cu (Sec. 2.3) on residues of three and four
// 64-bit words (wide.cuh): vadd, vsub, vmul (Barrett) and axpy (Shoup with the scalar's companion),
// one residue per thread step over a grid-stride loop.  Memory-bound like the narrower ones.
#include <cuda_runtime.h>

#include "common.cuh"
#include "wide.cuh"

namespace mq {
namespace {

constexpr int THREADS = 256;

template <int NL>
__device__ __forceinline__ Wide<NL> load(const void *p, size_t i) {
    const unsigned long long *s = reinterpret_cast<const unsigned long long *>(p) + NL * i;
    Wide<NL> r;
#pragma unroll
    for (int k = 0; k < NL; ++k) r.w[k] = __ldcs(s + k);
    return r;
}

template <int NL>
__device__ __forceinline__ void store(void *p, size_t i, const Wide<NL> &v) {
    unsigned long long *d = reinterpret_cast<unsigned long long *>(p) + NL * i;
#pragma unroll
    for (int k = 0; k < NL; ++k) __stcs(d + k, (unsigned long long)v.w[k]);
}

template <int NL, int OP>
__global__ void __launch_bounds__(THREADS) blas_wide_kernel(void *c, const void *a, const void *b, size_t n,
                                                            const ModW<NL> m, const Wide<NL> sc, const Wide<NL> scp) {
    for (size_t i = blockIdx.x * (size_t)THREADS + threadIdx.x; i < n; i += (size_t)gridDim.x * THREADS) {
        const Wide<NL> x = load<NL>(a, i), y = load<NL>(b, i);
        Wide<NL> r;
        if (OP == OP_VADD) r = add_mod(x, y, m.q);
        else if (OP == OP_VSUB) r = sub_mod(x, y, m.q);
        else if (OP == OP_VMUL) r = mul_mod_barrett(x, y, m);
        else r = add_mod(mul_mod_shoup(x, sc, scp, m.q), y, m.q);  // axpy: s*x + y with x = a, y = b
        store<NL>(c, i, r);
    }
}

template <int NL, int OP>
cudaError_t launch(const BlasWideArgs &a, cudaStream_t s) {
    ModW<NL> m;
    Wide<NL> sc, scp;
    for (int k = 0; k < NL; ++k) {
        m.q.w[k] = a.q[k];
        m.mu.w[k] = a.mu[k];
        sc.w[k] = a.s[k];
        scp.w[k] = a.sp[k];
    }
    m.L = a.L;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    size_t want = (a.n + THREADS - 1) / THREADS, cap = (size_t)(sms > 0 ? sms : 1) * 8;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    blas_wide_kernel<NL, OP><<<grid ? grid : 1, THREADS, 0, s>>>(a.c, a.a, a.b, a.n, m, sc, scp);
    return cudaGetLastError();
}

template <int NL>
cudaError_t launch_nl(int op, const BlasWideArgs &a, cudaStream_t s) {
    switch (op) {
    case OP_VADD: return launch<NL, OP_VADD>(a, s);
    case OP_VSUB: return launch<NL, OP_VSUB>(a, s);
    case OP_VMUL: return launch<NL, OP_VMUL>(a, s);
    case OP_AXPY: return launch<NL, OP_AXPY>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_blas_wide(int width, int op, const BlasWideArgs &a, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    if (width == 3) return launch_nl<3>(op, a, s);
    if (width == 4) return launch_nl<4>(op, a, s);
    return cudaErrorInvalidValue;
}

}  // namespace mq

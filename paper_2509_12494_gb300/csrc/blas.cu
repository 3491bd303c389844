// blas.cu -- element-wise modular BLAS over Z_q for sm_103a (Sec. 2.3: point-wise polynomial
// operations as vector add, vector subtract, point-wise vector multiply and axpy y = a x + y).
//
// Grid-stride kernels over 16-byte vectors: one 128-bit residue, or two 64-bit residues, per load.
// Every element is read once and written once by the same thread, so the output may alias either
// input.  Loads and stores carry the streaming (evict-first) hint: the vectors are read once.
// vmul uses Barrett reduction (general operands); axpy uses Shoup's method because its multiplier is
// one fixed scalar.  Both return the same canonical residue as any exact method.
#include <cuda_runtime.h>

#include "blas_ops.cuh"
#include "common.cuh"

namespace mq {
namespace {

constexpr int BLAS_THREADS = 256;
constexpr int BLAS_UNROLL = 4;  // 16-byte vectors in flight per thread and iteration

__host__ __device__ __forceinline__ uint4 u4(const uint64_t v[2]) {
    return make_uint4((uint32_t)v[0], (uint32_t)(v[0] >> 32), (uint32_t)v[1], (uint32_t)(v[1] >> 32));
}

template <int OP>
__global__ void __launch_bounds__(BLAS_THREADS) blas128_kernel(uint4 *c, const uint4 *a, const uint4 *b,
                                                               size_t n, const Mod128 m, const uint4 s, const uint4 sp) {
    const size_t stride = (size_t)gridDim.x * BLAS_THREADS * BLAS_UNROLL;
    for (size_t base = (size_t)blockIdx.x * BLAS_THREADS * BLAS_UNROLL + threadIdx.x; base < n; base += stride) {
        uint4 va[BLAS_UNROLL], vb[BLAS_UNROLL];
#pragma unroll
        for (int u = 0; u < BLAS_UNROLL; ++u) {
            size_t i = base + (size_t)u * BLAS_THREADS;
            if (i < n) {
                va[u] = __ldcs(a + i);
                vb[u] = __ldcs(b + i);
            }
        }
#pragma unroll
        for (int u = 0; u < BLAS_UNROLL; ++u) {
            size_t i = base + (size_t)u * BLAS_THREADS;
            if (i < n) __stcs(c + i, op128<OP>(va[u], vb[u], m, s, sp));
        }
    }
}

// 64-bit residues, two per 16-byte vector; `nv` vectors, then a scalar tail of `n` residues.
template <int OP>
__global__ void __launch_bounds__(BLAS_THREADS) blas64_kernel(uint64_t *c, const uint64_t *a,
                                                              const uint64_t *b, size_t n, const Mod64 m,
                                                              const uint64_t s, const uint64_t sp, int vec) {
    const size_t nt = (size_t)gridDim.x * BLAS_THREADS;
    const size_t tid = (size_t)blockIdx.x * BLAS_THREADS + threadIdx.x;
    size_t done = 0;
    if (vec) {
        const size_t nv = n / 2;
        const ulonglong2 *a2 = reinterpret_cast<const ulonglong2 *>(a), *b2 = reinterpret_cast<const ulonglong2 *>(b);
        ulonglong2 *c2 = reinterpret_cast<ulonglong2 *>(c);
        const size_t stride = nt * BLAS_UNROLL;
        for (size_t base = (size_t)blockIdx.x * BLAS_THREADS * BLAS_UNROLL + threadIdx.x; base < nv; base += stride) {
            ulonglong2 va[BLAS_UNROLL], vb[BLAS_UNROLL];
#pragma unroll
            for (int u = 0; u < BLAS_UNROLL; ++u) {
                size_t i = base + (size_t)u * BLAS_THREADS;
                if (i < nv) {
                    va[u] = __ldcs(a2 + i);
                    vb[u] = __ldcs(b2 + i);
                }
            }
#pragma unroll
            for (int u = 0; u < BLAS_UNROLL; ++u) {
                size_t i = base + (size_t)u * BLAS_THREADS;
                if (i < nv) {
                    ulonglong2 r;
                    r.x = op64<OP>(va[u].x, vb[u].x, m, s, sp);
                    r.y = op64<OP>(va[u].y, vb[u].y, m, s, sp);
                    __stcs(c2 + i, r);
                }
            }
        }
        done = nv * 2;
    }
    for (size_t i = done + tid; i < n; i += nt) c[i] = op64<OP>(a[i], b[i], m, s, sp);
}

// One wave: at most the CTAs of the kernel (width W, op OP) that are resident at once on the device
// (looked up once per kernel), so that no CTA waits for a second wave and the grid-stride loop
// covers the rest.
template <int W, int OP>
unsigned blas_grid(size_t work) {
    static int per_sm = 0, sms = 0;  // benign race: every thread computes the same values
    if (per_sm == 0) {
        int dev = 0, n = 0, m = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev);
        const cudaError_t e = W == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, blas128_kernel<OP>, BLAS_THREADS, 0)
                                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, blas64_kernel<OP>, BLAS_THREADS, 0);
        if (e != cudaSuccess || n < 1) n = 1;
        sms = m > 0 ? m : 1;
        per_sm = n;
    }
    const size_t per_block = (size_t)BLAS_THREADS * BLAS_UNROLL;
    size_t want = (work + per_block - 1) / per_block;
    const size_t cap = (size_t)sms * per_sm;
    if (want > cap) want = cap;
    return want ? (unsigned)want : 1u;
}

template <int OP>
cudaError_t launch_op(int width, const BlasArgs &a, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    if (width == 2) {
        Mod128 m{u4(a.q), u4(a.mu), a.L};
        blas128_kernel<OP><<<blas_grid<2, OP>(a.n), BLAS_THREADS, 0, s>>>(
            (uint4 *)a.c, (const uint4 *)a.a, (const uint4 *)a.b, a.n, m, u4(a.s), u4(a.sp));
    } else {
        Mod64 m{a.q[0], a.mu[0], a.L};
        int vec = ((((uintptr_t)a.a) | ((uintptr_t)a.b) | ((uintptr_t)a.c)) & 15) == 0;
        blas64_kernel<OP><<<blas_grid<1, OP>(vec ? a.n / 2 : a.n), BLAS_THREADS, 0, s>>>(
            (uint64_t *)a.c, (const uint64_t *)a.a, (const uint64_t *)a.b, a.n, m, a.s[0], a.sp[0], vec);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_blas(int width, int op, const BlasArgs &a, cudaStream_t s) {
    switch (op) {
    case OP_VADD: return launch_op<OP_VADD>(width, a, s);
    case OP_VSUB: return launch_op<OP_VSUB>(width, a, s);
    case OP_VMUL: return launch_op<OP_VMUL>(width, a, s);
    case OP_AXPY: return launch_op<OP_AXPY>(width, a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace mq

// mulvar.cu -- the general 124-bit modular product (Barrett) with either form of the double-word
// product: schoolbook (Eq. 8, the library's) or Karatsuba (Eq. 9).  Element-wise for parity tests,
// and as a throughput probe on register-resident operands, so the two can be compared where the
// multiply pipe, not memory, is the limit.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mqntt.h"
#include "../../include/mqntt_probe.h"
#include "hostmath.h"
#include "karatsuba.cuh"

int mq_cuda_fail(cudaError_t e, const char *where);
int mq_fail(int code, const char *fmt, ...);
int mq_check_modulus(const uint64_t q[2], int width, hm::u128 *qv);

namespace {

using namespace mq;

__device__ __forceinline__ uint4 ld4(const void *p, size_t i) { return reinterpret_cast<const uint4 *>(p)[i]; }

template <int V>
__device__ __forceinline__ uint4 mulmod(uint4 a, uint4 b, const Mod128 &m) {
    return V == MQ_MUL_KARATSUBA ? mul_mod_barrett_karatsuba(a, b, m) : mul_mod_barrett(a, b, m);
}

template <int V>
__global__ void mulvar_kernel(uint4 *c, const void *a, const void *b, size_t n, const Mod128 m) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        c[i] = mulmod<V>(ld4(a, i), ld4(b, i), m);
}

constexpr int RATE_THREADS = 256;
constexpr int RATE_CHAINS = 4;  // independent products in flight per thread

// v with every bit at position >= nbits cleared
__device__ __forceinline__ uint4 low_bits(uint4 v, int nbits) {
    uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int keep = nbits - 32 * i;
        w[i] = keep >= 32 ? w[i] : (keep <= 0 ? 0u : (w[i] & ((1u << keep) - 1u)));
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// Each thread runs RATE_CHAINS dependent chains x <- x * y mod q on operands below 2^(L-1) <= q.
template <int V>
__global__ void __launch_bounds__(RATE_THREADS) mulvar_rate_kernel(uint4 *out, int iters, const Mod128 m, uint4 seed) {
    uint4 x[RATE_CHAINS], y[RATE_CHAINS];
#pragma unroll
    for (int k = 0; k < RATE_CHAINS; ++k) {
        const uint32_t t = blockIdx.x * RATE_THREADS + threadIdx.x + 977u * k;
        x[k] = low_bits(make_uint4(seed.x ^ t, seed.y + t, seed.z * (t | 1u), seed.w ^ (t << 3)), m.L - 1);
        y[k] = low_bits(make_uint4(seed.w + 7u * t, seed.z ^ t, seed.y + k, seed.x + t), m.L - 1);
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < RATE_CHAINS; ++k) x[k] = mulmod<V>(x[k], y[k], m);
    }
    uint4 r = x[0];
#pragma unroll
    for (int k = 1; k < RATE_CHAINS; ++k) r = make_uint4(r.x ^ x[k].x, r.y ^ x[k].y, r.z ^ x[k].z, r.w ^ x[k].w);
    out[blockIdx.x * RATE_THREADS + threadIdx.x] = r;
}

int make_mod(const uint64_t q[2], Mod128 *m) {
    hm::u128 Q;
    int rc = mq_check_modulus(q, MQ_W128, &Q);
    if (rc) return rc;
    const int L = hm::bitlen(Q);
    uint64_t mu[2];
    hm::to_words(hm::barrett_mu(Q, L), mu);
    m->q = make_uint4((uint32_t)q[0], (uint32_t)(q[0] >> 32), (uint32_t)q[1], (uint32_t)(q[1] >> 32));
    m->mu = make_uint4((uint32_t)mu[0], (uint32_t)(mu[0] >> 32), (uint32_t)mu[1], (uint32_t)(mu[1] >> 32));
    m->L = L;
    return MQ_OK;
}

}  // namespace

extern "C" int mq_probe_mulmod(int variant, void *c, const void *a, const void *b, size_t n, const uint64_t q[2],
                               void *stream) {
    if (variant != MQ_MUL_SCHOOLBOOK && variant != MQ_MUL_KARATSUBA)
        return mq_fail(MQ_ERR_ARG, "unknown product variant %d", variant);
    Mod128 m;
    int rc = make_mod(q, &m);
    if (rc) return rc;
    if (n == 0) return MQ_OK;
    if (!c || !a || !b) return mq_fail(MQ_ERR_ARG, "NULL vector");
    if (((uintptr_t)c | (uintptr_t)a | (uintptr_t)b) & 15) return mq_fail(MQ_ERR_ALIGN, "vectors must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned blocks = (unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    if (variant == MQ_MUL_KARATSUBA) mulvar_kernel<MQ_MUL_KARATSUBA><<<blocks, 256, 0, s>>>((uint4 *)c, a, b, n, m);
    else mulvar_kernel<MQ_MUL_SCHOOLBOOK><<<blocks, 256, 0, s>>>((uint4 *)c, a, b, n, m);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MQ_OK : mq_cuda_fail(e, "product probe launch");
}

extern "C" int mq_probe_mulmod_rate(int variant, int iters, const uint64_t q[2], double *mulmod_per_s, double *ms,
                                    void *stream) {
    if (variant != MQ_MUL_SCHOOLBOOK && variant != MQ_MUL_KARATSUBA)
        return mq_fail(MQ_ERR_ARG, "unknown product variant %d", variant);
    if (iters <= 0 || !mulmod_per_s) return mq_fail(MQ_ERR_ARG, "iters must be positive and mulmod_per_s non-NULL");
    Mod128 m;
    int rc = make_mod(q, &m);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (variant == MQ_MUL_KARATSUBA)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mulvar_rate_kernel<MQ_MUL_KARATSUBA>, RATE_THREADS, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mulvar_rate_kernel<MQ_MUL_SCHOOLBOOK>, RATE_THREADS, 0);
    if (per_sm < 1) per_sm = 1;
    const int blocks = sms * per_sm;
    uint4 *out = nullptr;
    cudaError_t e = cudaMalloc(&out, (size_t)blocks * RATE_THREADS * sizeof(uint4));
    if (e != cudaSuccess) return mq_cuda_fail(e, "probe buffer");
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    const uint4 seed = make_uint4(0x9E3779B9u, 0x7F4A7C15u, 0x85EBCA6Bu, 0xC2B2AE35u);
    auto launch = [&](int n) {
        if (variant == MQ_MUL_KARATSUBA) mulvar_rate_kernel<MQ_MUL_KARATSUBA><<<blocks, RATE_THREADS, 0, s>>>(out, n, m, seed);
        else mulvar_rate_kernel<MQ_MUL_SCHOOLBOOK><<<blocks, RATE_THREADS, 0, s>>>(out, n, m, seed);
    };
    launch(1);  // warm-up
    cudaEventRecord(t0, s);
    launch(iters);
    cudaEventRecord(t1, s);
    e = cudaEventSynchronize(t1);
    float dt = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&dt, t0, t1);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFree(out);
    if (e != cudaSuccess) return mq_cuda_fail(e, "product probe");
    *mulmod_per_s = (double)blocks * RATE_THREADS * RATE_CHAINS * iters / (dt * 1e-3);
    if (ms) *ms = dt;
    return MQ_OK;
}

// ntt.cu -- twiddle-table construction and the dispatch of transform passes to the kernels
// instantiated in ntt_w{64,128}_{fwd,inv}.cu (the kernels themselves are in ntt_kernel.cuh).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "wide.cuh"

namespace mq {

// The driver's tensor-map encoder, looked up once through the runtime (no link to libcuda).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) == cudaSuccess &&
            qr == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Tensor map of one side of a TMA pass over 128-bit residues with tiles of 2^8 (tma.cuh):
//   column view: dims (2 N2 words of a row, N1 rows, batch), strides (16 N2, 16 stride) bytes,
//     box 16 words x 256 rows -- element l of 8 adjacent columns per 128-byte row;
//   row view: dims (16 words, N / 8 rows of 128 bytes, batch), strides (128, 16 stride), box
//     16 words x 256 rows -- 8 consecutive rows of 2^8 residues.
// Both with the 128-byte swizzle.  Returns 0, or nonzero when the map cannot be made.
int tile_map(CUtensorMap *m, bool col, const void *base, int logN, int L1, unsigned long long batch, size_t stride) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return -1;
    const int L2 = logN - L1;
    cuuint64_t dims[3], strides[2];
    cuuint32_t box[3] = {16, 256, 1}, es[3] = {1, 1, 1};
    if (col) {
        dims[0] = 2ull << L2;
        dims[1] = 1ull << L1;
        strides[0] = (1ull << L2) * 16;
    } else {
        dims[0] = 16;
        dims[1] = (1ull << logN) / 8;
        strides[0] = 128;
    }
    dims[2] = batch;
    strides[1] = (cuuint64_t)stride * 16;
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<void *>(base), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : (int)r;
}

cudaError_t launch_ntt_w3_fwd(int L, const PassArgs &a, cudaStream_t s);
cudaError_t launch_ntt_w3_inv(int L, const PassArgs &a, cudaStream_t s);
cudaError_t launch_ntt_w4_fwd(int L, const PassArgs &a, cudaStream_t s);
cudaError_t launch_ntt_w4_inv(int L, const PassArgs &a, cudaStream_t s);
cudaError_t launch_ntt_w1_fwd(int L, const PassArgs &a, cudaStream_t s);
cudaError_t launch_ntt_w1_inv(int L, const PassArgs &a, cudaStream_t s);
cudaError_t launch_ntt_w2_fwd(int L, const PassArgs &a, cudaStream_t s);
cudaError_t launch_ntt_w2_inv(int L, const PassArgs &a, cudaStream_t s);

namespace {

__device__ __forceinline__ unsigned brv(unsigned v, int bits) { return bits ? (__brev(v) >> (32 - bits)) : 0u; }

// ------------------------------------------------------------------------------------------------
// twiddle tables
// ------------------------------------------------------------------------------------------------

__device__ uint64_t shoup_companion(uint64_t w, uint64_t q) {  // floor(w * 2^64 / q), w < q < 2^63
    uint64_t r = w, quo = 0;
    for (int i = 0; i < 64; ++i) {
        r <<= 1;
        uint64_t bit = r >= q;
        r -= bit ? q : 0;
        quo = (quo << 1) | bit;
    }
    return quo;
}

__device__ uint4 shl1(uint4 v) {
    return make_uint4(v.x << 1, (v.y << 1) | (v.x >> 31), (v.z << 1) | (v.y >> 31), (v.w << 1) | (v.z >> 31));
}

__device__ uint4 shoup_companion(uint4 w, uint4 q) {  // floor(w * 2^128 / q), w < q < 2^127
    uint4 r = w, quo = make_uint4(0, 0, 0, 0);
    for (int i = 0; i < 128; ++i) {
        r = shl1(r);
        uint32_t m;
        uint4 d = sub128(r, q, m);
        r = sel128(m, r, d);
        quo = shl1(quo);
        quo.x |= (~m) & 1u;
    }
    return quo;
}

__device__ uint64_t pow_mod(uint64_t g, unsigned e, const Mod64 &m) {
    uint64_t acc = 1 % m.q;
    for (int b = 31; b >= 0; --b) {
        acc = mul_mod_barrett(acc, acc, m);
        if ((e >> b) & 1) acc = mul_mod_barrett(acc, g, m);
    }
    return acc;
}

__device__ uint4 pow_mod(uint4 g, unsigned e, const Mod128 &m) {
    uint4 acc = make_uint4(1, 0, 0, 0);
    for (int b = 31; b >= 0; --b) {
        acc = mul_mod_barrett(acc, acc, m);
        if ((e >> b) & 1) acc = mul_mod_barrett(acc, g, m);
    }
    return acc;
}

__device__ __forceinline__ unsigned table_exponent(unsigned k, int logN, int cyclic) {
    if (k == 0) return 0;
    if (!cyclic) return brv(k, logN);
    unsigned m = 1u << (31 - __clz(k));
    return brv(k - m, logN - 1);
}

__global__ void twiddle_kernel64(int logN, int cyclic, Mod64 m, uint64_t root, uint64_t root_inv, Tw64 *fwd, Tw64 *inv) {
    unsigned N = 1u << logN;
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        unsigned e = table_exponent(k, logN, cyclic);
        uint64_t w = pow_mod(root, e, m), wi = pow_mod(root_inv, e, m);
        fwd[k] = Tw64{w, shoup_companion(w, m.q)};
        inv[k] = Tw64{wi, shoup_companion(wi, m.q)};
    }
}

__global__ void twiddle_kernel128(int logN, int cyclic, Mod128 m, uint4 root, uint4 root_inv, Tw128 *fwd, Tw128 *inv) {
    unsigned N = 1u << logN;
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        unsigned e = table_exponent(k, logN, cyclic);
        uint4 w = pow_mod(root, e, m), wi = pow_mod(root_inv, e, m);
        Tw128 f, v;
        f.w = w;
        f.wp = shoup_companion(w, m.q);
        v.w = wi;
        v.wp = shoup_companion(wi, m.q);
        fwd[k] = f;
        inv[k] = v;
    }
}

// residues of three and four words (wide.cuh): the same tables, entries of 2 NL words (w, w')
template <int NL>
__device__ Wide<NL> shoup_companion(const Wide<NL> &w, const Wide<NL> &q) {  // floor(w 2^(64 NL) / q), q < 2^(64 NL - 4)
    Wide<NL> r = w, quo;
#pragma unroll
    for (int k = 0; k < NL; ++k) quo.w[k] = 0;
    for (int i = 0; i < 64 * NL; ++i) {
        r = add_nored(r, r);
        quo = add_nored(quo, quo);
        uint64_t br;
        const Wide<NL> d = sub_wide(r, q, br);
        if (!br) {
            r = d;
            quo.w[0] |= 1;
        }
    }
    return quo;
}

template <int NL>
__device__ Wide<NL> pow_mod(const Wide<NL> &g, unsigned e, const ModW<NL> &m) {
    Wide<NL> acc;
#pragma unroll
    for (int k = 0; k < NL; ++k) acc.w[k] = k == 0;
    for (int b = 31; b >= 0; --b) {
        acc = mul_mod_barrett(acc, acc, m);
        if ((e >> b) & 1) acc = mul_mod_barrett(acc, g, m);
    }
    return acc;
}

template <int NL>
__global__ void twiddle_kernel_wide(int logN, int cyclic, ModW<NL> m, Wide<NL> root, Wide<NL> root_inv,
                                    uint64_t *fwd, uint64_t *inv) {
    unsigned N = 1u << logN;
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        unsigned e = table_exponent(k, logN, cyclic);
        const Wide<NL> w = pow_mod(root, e, m), wi = pow_mod(root_inv, e, m);
        const Wide<NL> wp = shoup_companion(w, m.q), wip = shoup_companion(wi, m.q);
#pragma unroll
        for (int j = 0; j < NL; ++j) {
            fwd[2 * NL * (size_t)k + j] = w.w[j];
            fwd[2 * NL * (size_t)k + NL + j] = wp.w[j];
            inv[2 * NL * (size_t)k + j] = wi.w[j];
            inv[2 * NL * (size_t)k + NL + j] = wip.w[j];
        }
    }
}

template <int NL>
void launch_twiddles_wide(int logN, int cyclic, const uint64_t *q, const uint64_t *root, const uint64_t *root_inv,
                          const uint64_t *mu, int L, void *tw_fwd, void *tw_inv, unsigned blocks, unsigned threads,
                          cudaStream_t s) {
    ModW<NL> m;
    Wide<NL> r, ri;
    for (int k = 0; k < NL; ++k) {
        m.q.w[k] = q[k];
        m.mu.w[k] = mu[k];
        r.w[k] = root[k];
        ri.w[k] = root_inv[k];
    }
    m.L = L;
    twiddle_kernel_wide<NL><<<blocks, threads, 0, s>>>(logN, cyclic, m, r, ri, (uint64_t *)tw_fwd, (uint64_t *)tw_inv);
}

uint4 to_u4(const uint64_t v[2]) {
    return make_uint4((uint32_t)v[0], (uint32_t)(v[0] >> 32), (uint32_t)v[1], (uint32_t)(v[1] >> 32));
}

}  // namespace

cudaError_t launch_ntt_pass(int width, int L, bool inv, const PassArgs &a, cudaStream_t s) {
    if (width == 1) return inv ? launch_ntt_w1_inv(L, a, s) : launch_ntt_w1_fwd(L, a, s);
    if (width == 3) return inv ? launch_ntt_w3_inv(L, a, s) : launch_ntt_w3_fwd(L, a, s);
    if (width == 4) return inv ? launch_ntt_w4_inv(L, a, s) : launch_ntt_w4_fwd(L, a, s);
    return inv ? launch_ntt_w2_inv(L, a, s) : launch_ntt_w2_fwd(L, a, s);
}

cudaError_t launch_twiddle_build(int width, int logN, int cyclic, const uint64_t q[2], const uint64_t root[2],
                                 const uint64_t root_inv[2], const uint64_t mu[2], int L, void *tw_fwd,
                                 void *tw_inv, cudaStream_t s) {
    unsigned N = 1u << logN;
    unsigned threads = 256, blocks = (N + threads - 1) / threads;
    if (width == 1) {
        Mod64 m{q[0], mu[0], L};
        twiddle_kernel64<<<blocks, threads, 0, s>>>(logN, cyclic, m, root[0], root_inv[0], (Tw64 *)tw_fwd, (Tw64 *)tw_inv);
    } else if (width == 3) {
        launch_twiddles_wide<3>(logN, cyclic, q, root, root_inv, mu, L, tw_fwd, tw_inv, blocks, threads, s);
    } else if (width == 4) {
        launch_twiddles_wide<4>(logN, cyclic, q, root, root_inv, mu, L, tw_fwd, tw_inv, blocks, threads, s);
    } else {
        Mod128 m{to_u4(q), to_u4(mu), L};
        twiddle_kernel128<<<blocks, threads, 0, s>>>(logN, cyclic, m, to_u4(root), to_u4(root_inv), (Tw128 *)tw_fwd,
                                                     (Tw128 *)tw_inv);
    }
    return cudaGetLastError();
}

}  // namespace mq

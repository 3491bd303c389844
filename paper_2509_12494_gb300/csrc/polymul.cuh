// polymul.cuh -- the fused pass of the polynomial product through the NTT (Sec. 2.3): the last
// forward stages of both operands, their pointwise product and the first inverse stages in one
// kernel, on tiles of 2^L residues held in shared memory.
//
// For N <= 2^12 (one pass) this is the whole product: a CTA stages a group of a's and b's
// polynomials, transforms both (forward, bit-reversed order in the tile), multiplies them pointwise
// and transforms the product back (inverse, N^-1 folded in), and stores canonical coefficients.  For
// larger N the column passes run as ordinary pass launches before (forward, a and b) and after
// (inverse) this kernel, which then works on rows: forward row stages of both, product, inverse row
// stages, lazy residues stored for the inverse column pass.
#pragma once
#include "ntt_kernel.cuh"

namespace mq {
namespace polymul_detail {

using ntt_detail::Shape;
using ntt_detail::Traits;

template <int W>
struct ModOf;
template <>
struct ModOf<1> {
    typedef Mod64 M;
    __device__ __forceinline__ static M make(const MulArgs &m) { return Mod64{m.q[0], m.mu[0], m.L}; }
};
template <>
struct ModOf<2> {
    typedef Mod128 M;
    __device__ __forceinline__ static M make(const MulArgs &m) {
        return Mod128{Traits<2>::make(m.q), Traits<2>::make(m.mu), m.L};
    }
};

// fa / fb: the forward pass over a's / b's tiles (their `in` is read); ia: the inverse pass whose
// `out` receives the product.  All three describe the same tiles (same shape, split and layout).
template <int W, int L>
__global__ void __launch_bounds__(Shape<W, L>::NT, (Shape<W, L>::NT <= 256) ? 3 : 1)
    polymul_kernel(const PassArgs fa, const PassArgs fb, const PassArgs ia, const MulArgs m,
                   unsigned long long groups) {
    typedef Traits<W> Tr;
    typedef typename Tr::E E;
    typedef Shape<W, L> S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    E *ta = reinterpret_cast<E *>(smem_raw), *tb = ta + S::G * S::TS;
    const int tid = threadIdx.x;
    for (unsigned long long grp = blockIdx.x; grp < groups; grp += gridDim.x) {
        const unsigned long long first = grp * S::G;
        ntt_detail::load_tiles_sync<W, L>(fa, first, ta, tid);
        ntt_detail::load_tiles_sync<W, L>(fb, first, tb, tid);
        __syncthreads();
        ntt_detail::tile_rounds<W, L, false>(fa, first, ta, tid);
        ntt_detail::tile_rounds<W, L, false>(fb, first, tb, tid);
        // pointwise product of the two spectra: canonical operands (forward values are below 16q),
        // Barrett product, canonical result -- the same arithmetic as mod_vmul
        {
            const E q = Tr::make(fa.q);
            const E q2 = add_nored(q, q);
            const E q4 = add_nored(q2, q2);
            const E q8 = add_nored(q4, q4);
            const typename ModOf<W>::M mod = ModOf<W>::make(m);
            for (int i = tid; i < S::G * S::T; i += S::NT) {
                const int at = (i / S::T) * S::TS + ntt_detail::swz<W>(i % S::T);
                const E x = csub(csub(csub(csub(ta[at], q8), q4), q2), q);
                const E y = csub(csub(csub(csub(tb[at], q8), q4), q2), q);
                ta[at] = mul_mod_barrett(x, y, mod);
            }
        }
        __syncthreads();
        ntt_detail::tile_compute_store<W, L, true>(ia, first, ta, tid);  // ends with a barrier
    }
}

template <int W, int L>
cudaError_t launch_polymul_one(const PassArgs &fa, const PassArgs &fb, const PassArgs &ia, const MulArgs &m,
                               cudaStream_t s) {
    typedef Shape<W, L> S;
    static int per_sm = 0;  // benign race: every thread computes the same values
    const size_t smem = 2 * S::SMEM;
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(polymul_kernel<W, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, polymul_kernel<W, L>, S::NT, smem);
        if (e != cudaSuccess) return e;
        per_sm = n > 0 ? n : 1;
    }
    const unsigned long long TP = ia.col ? (1ull << (ia.logN - ia.L1)) : (1ull << ia.L1);
    const unsigned long long groups = (TP * ia.batch + S::G - 1) / S::G;
    if (groups == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned long long wave = (unsigned long long)sms * per_sm;
    polymul_kernel<W, L><<<(unsigned)(groups < wave ? groups : wave), S::NT, smem, s>>>(fa, fb, ia, m, groups);
    return cudaGetLastError();
}

template <int W>
cudaError_t launch_polymul_w(int L, const PassArgs &fa, const PassArgs &fb, const PassArgs &ia, const MulArgs &m,
                             cudaStream_t s) {
    switch (L) {
    case 1: return launch_polymul_one<W, 1>(fa, fb, ia, m, s);
    case 2: return launch_polymul_one<W, 2>(fa, fb, ia, m, s);
    case 3: return launch_polymul_one<W, 3>(fa, fb, ia, m, s);
    case 4: return launch_polymul_one<W, 4>(fa, fb, ia, m, s);
    case 5: return launch_polymul_one<W, 5>(fa, fb, ia, m, s);
    case 6: return launch_polymul_one<W, 6>(fa, fb, ia, m, s);
    case 7: return launch_polymul_one<W, 7>(fa, fb, ia, m, s);
    case 8: return launch_polymul_one<W, 8>(fa, fb, ia, m, s);
    case 9: return launch_polymul_one<W, 9>(fa, fb, ia, m, s);
    case 10: return launch_polymul_one<W, 10>(fa, fb, ia, m, s);
    case 11: return launch_polymul_one<W, 11>(fa, fb, ia, m, s);
    case 12: return launch_polymul_one<W, 12>(fa, fb, ia, m, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace polymul_detail
}  // namespace mq

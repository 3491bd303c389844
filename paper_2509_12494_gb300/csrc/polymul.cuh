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

// The same pass in the TMA form (128-bit residues, rows of 2^8, unpermuted row views, tma.cuh): a
// group's rows of a and of b arrive as two tensor copies on one mbarrier, the product leaves as one
// tensor store.  Both buffers hold operands, so there is no prefetch; the CTAs of an SM (three)
// overlap one another's copies and arithmetic.
template <int W>
__global__ void __launch_bounds__(256, 3)
    polymul_tma_kernel(const __grid_constant__ CUtensorMap ma, const __grid_constant__ CUtensorMap mb,
                       const __grid_constant__ CUtensorMap mc, const PassArgs fa, const PassArgs ia, const MulArgs m,
                       unsigned long long groups) {
    static_assert(W == 2, "the TMA form is that of 128-bit residues");
    typedef Traits<W> Tr;
    typedef typename Tr::E E;
    typedef Shape<W, TMA_L> S;
    constexpr unsigned B = ntt_detail::TMA_GROUP_BYTES;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_ok;
    const int tid = threadIdx.x;
    unsigned char *p = smem_raw + ((1024u - (tma::su32(smem_raw) & 1023u)) & 1023u);
    E *const ta = reinterpret_cast<E *>(p), *const tb = reinterpret_cast<E *>(p + B);
    const ntt_detail::TileAddr tadr(fa);
    if (tid == 0) {
        tma::mbar_init(&bar, 1);
        tma::mbar_init_fence();
    }
    __syncthreads();
    unsigned ph = 0;
    for (unsigned long long grp = blockIdx.x; grp < groups; grp += gridDim.x) {
        const unsigned long long first = grp * S::G;
        if (tid == 0) {
            int x, y, z;
            ntt_detail::tma_box(tadr, false, first, x, y, z);
            tma::store_wait_read();  // the previous group's store has read buffer a
            tma::mbar_expect(&bar, 2 * B);
            tma::load3(ta, &ma, x, y, z, &bar);
            tma::load3(tb, &mb, x, y, z, &bar);
            s_ok = tma::mbar_wait(&bar, ph, ntt_detail::TMA_WAIT_NS);
        }
        __syncthreads();
        if (!s_ok) {
            if (tid == 0) {  // record the fault, then wait (bounded again) for the copies in flight
                atomicCAS(&ntt_detail::g_tma_fault, 0ull, grp + 1);
                tma::mbar_wait(&bar, ph, ntt_detail::TMA_WAIT_NS);
            }
            break;
        }
        while (!tma::mbar_test(&bar, ph)) {  // completed: thread 0 saw it
        }
        ph ^= 1u;
        ntt_detail::tma_rounds<false, false>(fa, ta, first, tid);
        ntt_detail::tma_rounds<false, false>(fa, tb, first, tid);
        __syncthreads();
        {  // pointwise product of the canonicalised spectra (Barrett, as mod_vmul); the layouts match
            const E q = Tr::make(fa.q);
            const E q2 = add_nored(q, q), q4 = add_nored(q2, q2), q8 = add_nored(q4, q4);
            const typename ModOf<W>::M mod = ModOf<W>::make(m);
            for (int i = tid; i < S::G * S::T; i += S::NT) {
                const E x = csub(csub(csub(csub(ta[i], q8), q4), q2), q);
                const E y = csub(csub(csub(csub(tb[i], q8), q4), q2), q);
                ta[i] = mul_mod_barrett(x, y, mod);
            }
        }
        __syncthreads();
        ntt_detail::tma_rounds<true, false>(ia, ta, first, tid);
        tma::fence_async_shared();
        __syncthreads();
        if (tid == 0) {
            int x, y, z;
            ntt_detail::tma_box(tadr, false, first, x, y, z);
            tma::store3(&mc, x, y, z, ta);
            tma::store_commit();
        }
    }
    if (tid == 0) tma::store_wait();
}

// Launch the TMA form when every side qualifies; *taken = false otherwise (or when a map fails).
inline cudaError_t launch_polymul_tma(const PassArgs &fa, const PassArgs &fb, const PassArgs &ia, const MulArgs &m,
                                      cudaStream_t s, bool *taken) {
    *taken = false;
    PassArgs iv = ia;  // the inverse pass reads what the forward one staged: same view
    iv.in = ia.out;
    iv.in_stride = ia.out_stride;
    if (!tma_eligible(fa) || !tma_eligible(fb) || !tma_eligible(iv) || fa.col) return cudaSuccess;
    const unsigned long long groups = ntt_detail::pass_tiles(fa) / Shape<2, TMA_L>::G;
    if (groups < (unsigned long long)ntt_detail::sm_count()) return cudaSuccess;
    CUtensorMap ma, mb, mc;
    if (tile_map(&ma, false, fa.in, fa.logN, fa.L1, fa.batch, fa.in_stride) ||
        tile_map(&mb, false, fb.in, fb.logN, fb.L1, fb.batch, fb.in_stride) ||
        tile_map(&mc, false, ia.out, ia.logN, ia.L1, ia.batch, ia.out_stride))
        return cudaSuccess;
    static int per_sm = 0;  // benign race: every thread computes the same values
    const size_t smem = 2 * (size_t)ntt_detail::TMA_GROUP_BYTES + 1024;
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(polymul_tma_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, polymul_tma_kernel<2>, 256, smem);
        if (e != cudaSuccess) return e;
        per_sm = n > 0 ? n : 1;
    }
    const unsigned long long wave = (unsigned long long)ntt_detail::sm_count() * per_sm;
    polymul_tma_kernel<2><<<(unsigned)(groups < wave ? groups : wave), 256, smem, s>>>(ma, mb, mc, fa, ia, m, groups);
    *taken = true;
    return cudaGetLastError();
}

template <int W, int L>
cudaError_t launch_polymul_one(const PassArgs &fa, const PassArgs &fb, const PassArgs &ia, const MulArgs &m,
                               cudaStream_t s) {
    typedef Shape<W, L> S;
    if constexpr (W == 2 && L == TMA_L) {
        bool taken = false;
        cudaError_t e = launch_polymul_tma(fa, fb, ia, m, s, &taken);
        if (e != cudaSuccess || taken) return e;
    }
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

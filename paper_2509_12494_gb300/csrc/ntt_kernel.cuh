// ntt_kernel.cuh -- negacyclic / cyclic NTT kernels for sm_103a (instantiated by ntt_w*_*.cu).
//
// The transform is the in-place radix-2 Cooley-Tukey algorithm whose butterfly (Sec. 3.2, last
// paragraph: one modular add, one sub, one mul) runs over log2 N stages of N/2 butterflies.  The
// negacyclic twist psi^j is merged into the twiddles: the table holds psi^brv(k) (bit-reversed
// exponent), forward stage m uses entry m + i for butterfly group i, and the output comes out in
// bit-reversed order.  The inverse runs the stages backwards with Gentleman-Sande butterflies
// (u + v, (u - v) w^-1) on the table of psi^-brv(k) and folds N^-1 into the last stage.  The cyclic
// transform of Eq. 4 uses the same kernels with the table w^brv'(k) (brv' over log2 N - 1 bits of
// k minus its leading power of two).
//
// Work decomposition (GB300-first, not the paper's AVX-512 Pease dataflow):
//   * the N residues are viewed as an N1 x N2 matrix (N1 = 2^L1).  The first L1 forward stages only
//     mix residues of one column; the remaining ones only mix residues of one row.  A "column pass"
//     transforms whole columns, a "row pass" whole rows; N <= 2^12 needs one pass (N1 = 1);
//   * a CTA owns G tiles (columns or rows) staged in shared memory by a cooperative, coalesced copy
//     (G consecutive columns give G-residue contiguous segments in global memory);
//   * inside a tile each thread holds R = 8 residues in registers and runs 3 stages on them
//     (radix-8), then the tile is exchanged through shared memory for the next 3 stages;
//   * natural-order output (or input, for the inverse) is a bit-reversal permutation folded into
//     the row pass' global addresses, with tiles chosen so that every CTA still writes contiguous
//     segments; the two passes then go through a scratch buffer because the permutation is not
//     in place.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace mq {
namespace ntt_detail {

template <int W>
struct Traits;
template <>
struct Traits<1> {
    typedef uint64_t E;
    typedef Tw64 TW;
    static constexpr int EPR = 16;  // residues per 128-byte shared-memory row
    __device__ __forceinline__ static E make(const uint64_t v[2]) { return v[0]; }
    __device__ __forceinline__ static void load_tw(const TW *t, unsigned idx, E &w, E &wp) {
        ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(t) + idx);
        w = v.x;
        wp = v.y;
    }
};
template <>
struct Traits<2> {
    typedef uint4 E;
    typedef Tw128 TW;
    static constexpr int EPR = 8;
    __device__ __forceinline__ static E make(const uint64_t v[2]) {
        return make_uint4((uint32_t)v[0], (uint32_t)(v[0] >> 32), (uint32_t)v[1], (uint32_t)(v[1] >> 32));
    }
    __device__ __forceinline__ static void load_tw(const TW *t, unsigned idx, E &w, E &wp) {
        const uint4 *p = reinterpret_cast<const uint4 *>(t) + 2 * (size_t)idx;
        w = __ldg(p);
        wp = __ldg(p + 1);
    }
};

constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v >> 1); }
constexpr int maxc(int a, int b) { return a > b ? a : b; }

// Static shape of the kernel for tiles of 2^L residues.
template <int W, int L>
struct Shape {
    static constexpr int T = 1 << L;                 // residues per tile
    static constexpr int R = T < 8 ? T : 8;          // residues per thread (radix)
    static constexpr int r = ilog2c(R);              // stages per register round
    static constexpr int TPT = T / R;                // threads per tile
    static constexpr int G = (L <= 9) ? maxc(8, 256 / TPT) : (L == 10 ? 2 : 1);  // tiles per CTA
    static constexpr int NT = G * TPT;               // threads per CTA
    static constexpr int TS = T + 1;                 // padded tile stride in shared memory
    static constexpr int ROUNDS = (L + r - 1) / r;
    static constexpr size_t SMEM = (size_t)G * TS * sizeof(typename Traits<W>::E);
};

__device__ __forceinline__ unsigned brv(unsigned v, int bits) { return bits ? (__brev(v) >> (32 - bits)) : 0u; }

// XOR swizzle of a tile-local index inside its 128-byte row group, so that strided register
// rounds do not pile onto the same banks.
template <int W>
__device__ __forceinline__ int swz(int l) {
    constexpr int EPR = Traits<W>::EPR;
    return l ^ ((l / EPR) & (EPR - 1));
}

// Global residue index (within one polynomial) of element l of tile ti.
__device__ __forceinline__ size_t tile_pos(int layout, unsigned ti, unsigned l, int L, int L1, int logN, int perm) {
    const int L2 = logN - L1;
    if (layout == LAYOUT_COL) return ((size_t)l << L2) + ti;
    if (layout == LAYOUT_ROW) {
        unsigned h = perm ? brv(ti, L1) : ti;
        return ((size_t)h << L2) + l;
    }
    // LAYOUT_NAT: row h = brv_L1(ti) of the bit-reversed view, element l sits at brv_L(l) * N1 + ti
    return ((size_t)brv(l, L) << L1) + ti;
}

template <int W, int L, bool INV>
__global__ void __launch_bounds__(Shape<W, L>::NT, (Shape<W, L>::NT <= 256) ? 2 : 1) ntt_pass_kernel(const PassArgs a) {
    typedef Traits<W> Tr;
    typedef typename Tr::E E;
    typedef Shape<W, L> S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    E *sm = reinterpret_cast<E *>(smem_raw);

    const E q = Tr::make(a.q);
    const int L1 = a.L1, logN = a.logN;
    const unsigned TP = a.col ? (1u << (logN - L1)) : (1u << L1);  // tiles per polynomial
    const unsigned long long first_tile = (unsigned long long)blockIdx.x * S::G;
    const typename Tr::TW *tw = reinterpret_cast<const typename Tr::TW *>(a.tw);
    const E *in = reinterpret_cast<const E *>(a.in);
    E *out = reinterpret_cast<E *>(a.out);
    const bool gfast_in = a.in_layout != LAYOUT_ROW, gfast_out = a.out_layout != LAYOUT_ROW;

    // ---- global -> shared (coalesced: consecutive threads take consecutive global residues)
    for (int i = threadIdx.x; i < S::G * S::T; i += S::NT) {
        int g = gfast_in ? (i % S::G) : (i / S::T);
        int l = gfast_in ? (i / S::G) : (i % S::T);
        unsigned long long gt = first_tile + g;
        unsigned long long poly = gt / TP;
        unsigned ti = (unsigned)(gt % TP);
        E v;
        if (poly < a.batch)
            v = in[poly * a.in_stride + tile_pos(a.in_layout, ti, l, L, L1, logN, a.perm)];
        else
            v = E();
        sm[g * S::TS + swz<W>(l)] = v;
    }
    __syncthreads();

    // ---- register rounds of up to three stages
    const int g = threadIdx.x / S::TPT, t = threadIdx.x % S::TPT;
    unsigned tw_base;
    {
        unsigned long long gt = first_tile + g;
        unsigned ti = (unsigned)(gt % TP);
        tw_base = a.col ? 1u : ((1u << L1) + (a.perm ? brv(ti, L1) : ti));
    }
    E *tile = sm + g * S::TS;
    E x[S::R];

#pragma unroll
    for (int rr_ = 0; rr_ < S::ROUNDS; ++rr_) {
        const int rho = INV ? (S::ROUNDS - 1 - rr_) : rr_;
        const int s_begin = rho * S::r;
        const int s_end = (s_begin + S::r < L) ? s_begin + S::r : L;
        const int rr = s_end - s_begin;  // stages in this round
        const int b_hi = L - 1 - s_begin, b_lo = L - s_end;
        const int V = S::R >> rr;        // independent groups per thread in this round
        int base[S::R];
#pragma unroll
        for (int k = 0; k < V; ++k) {
            int vt = t + k * S::TPT;
            int lo = vt & ((1 << b_lo) - 1), hi = vt >> b_lo;
            base[k] = (hi << (b_hi + 1)) | lo;
#pragma unroll
            for (int e = 0; e < (1 << rr); ++e) x[k * (1 << rr) + e] = tile[swz<W>(base[k] | (e << b_lo))];
        }
#pragma unroll
        for (int jj = 0; jj < rr; ++jj) {
            const int j = INV ? (rr - 1 - jj) : jj;
            const int s = s_begin + j;                 // local stage
            const int half = 1 << (rr - 1 - j);        // distance in the register index
#pragma unroll
            for (int k = 0; k < V; ++k) {
#pragma unroll
                for (int e0 = 0; e0 < (1 << rr); ++e0) {
                    if (e0 & half) continue;
                    const int l0 = base[k] | (e0 << b_lo);
                    const unsigned idx = (tw_base << s) + ((unsigned)l0 >> (L - s));
                    E &u = x[k * (1 << rr) + e0];
                    E &v = x[k * (1 << rr) + e0 + half];
                    E w, wp;
                    if (!INV) {
                        Tr::load_tw(tw, idx, w, wp);
                        E tv = mul_mod_shoup(v, w, wp, q);
                        E nu = add_mod(u, tv, q);
                        v = sub_mod(u, tv, q);
                        u = nu;
                    } else if (s == 0 && a.scale) {
                        E sum = add_mod(u, v, q), dif = sub_mod(u, v, q);
                        u = mul_mod_shoup(sum, Tr::make(a.sc), Tr::make(a.scp), q);
                        v = mul_mod_shoup(dif, Tr::make(a.ws), Tr::make(a.wsp), q);
                    } else {
                        Tr::load_tw(tw, idx, w, wp);
                        E sum = add_mod(u, v, q), dif = sub_mod(u, v, q);
                        u = sum;
                        v = mul_mod_shoup(dif, w, wp, q);
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < V; ++k) {
#pragma unroll
            for (int e = 0; e < (1 << rr); ++e) tile[swz<W>(base[k] | (e << b_lo))] = x[k * (1 << rr) + e];
        }
        __syncthreads();
    }

    // ---- shared -> global
    for (int i = threadIdx.x; i < S::G * S::T; i += S::NT) {
        int gg = gfast_out ? (i % S::G) : (i / S::T);
        int l = gfast_out ? (i / S::G) : (i % S::T);
        unsigned long long gt = first_tile + gg;
        unsigned long long poly = gt / TP;
        unsigned ti = (unsigned)(gt % TP);
        if (poly < a.batch)
            out[poly * a.out_stride + tile_pos(a.out_layout, ti, l, L, L1, logN, a.perm)] = sm[gg * S::TS + swz<W>(l)];
    }
}

template <int W, int L, bool INV>
cudaError_t launch_one(const PassArgs &a, cudaStream_t s) {
    typedef Shape<W, L> S;
    static bool configured = false;  // benign race: every thread sets the same attribute
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(ntt_pass_kernel<W, L, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)S::SMEM);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const unsigned long long TP = a.col ? (1ull << (a.logN - a.L1)) : (1ull << a.L1);
    const unsigned long long tiles = TP * a.batch;
    const unsigned long long grid = (tiles + S::G - 1) / S::G;
    if (grid == 0) return cudaSuccess;
    if (grid > 0x7fffffffull) return cudaErrorInvalidConfiguration;
    ntt_pass_kernel<W, L, INV><<<(unsigned)grid, S::NT, S::SMEM, s>>>(a);
    return cudaGetLastError();
}

template <int W, bool INV>
cudaError_t launch_w(int L, const PassArgs &a, cudaStream_t s) {
    switch (L) {
    case 1: return launch_one<W, 1, INV>(a, s);
    case 2: return launch_one<W, 2, INV>(a, s);
    case 3: return launch_one<W, 3, INV>(a, s);
    case 4: return launch_one<W, 4, INV>(a, s);
    case 5: return launch_one<W, 5, INV>(a, s);
    case 6: return launch_one<W, 6, INV>(a, s);
    case 7: return launch_one<W, 7, INV>(a, s);
    case 8: return launch_one<W, 8, INV>(a, s);
    case 9: return launch_one<W, 9, INV>(a, s);
    case 10: return launch_one<W, 10, INV>(a, s);
    case 11: return launch_one<W, 11, INV>(a, s);
    case 12: return launch_one<W, 12, INV>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ntt_detail
}  // namespace mq

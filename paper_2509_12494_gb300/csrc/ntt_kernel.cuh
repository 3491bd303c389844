// ntt_kernel.cuh -- negacyclic / cyclic NTT kernels for sm_103a (instantiated by ntt_w*_*.cu).
//
// The transform is the in-place radix-2 Cooley-Tukey algorithm whose butterfly (Sec. 3.2, last
// paragraph: one modular add, one sub, one mul) runs over log2 N stages of N/2 butterflies.  The
// negacyclic twist psi^j is merged into the twiddles: the table holds psi^brv(k) (bit-reversed
// exponent), forward stage m uses entry m + i for butterfly group i, and the output comes out in
// bit-reversed order.  The inverse runs the stages backwards with Gentleman-Sande butterflies
// (u + v, (u - v) w^-1) on the table of psi^-brv(k) and folds N^-1 into the last stage.  The cyclic
// transform of Eq. 11 uses the same kernels with the table w^brv'(k) (brv' over log2 N - 1 bits of
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
//   * a pass too small to give every SM a CTA takes the latency shape instead: one tile per CTA,
//     R = 4 (radix-4 rounds on more threads), the tile's twiddles staged in shared memory;
//   * natural-order output (or input, for the inverse) is a bit-reversal permutation folded into
//     the row pass' global addresses, with tiles chosen so that every CTA still writes contiguous
//     segments; the two passes then go through a scratch buffer because the permutation is not
//     in place.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"
#include "tma.cuh"
#include "wide.cuh"

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
    __device__ __forceinline__ static void load_tw_shared(const TW *t, unsigned idx, E &w, E &wp) {
        ulonglong2 v = reinterpret_cast<const ulonglong2 *>(t)[idx];
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
    __device__ __forceinline__ static void load_tw_shared(const TW *t, unsigned idx, E &w, E &wp) {
        const uint4 *p = reinterpret_cast<const uint4 *>(t) + 2 * idx;
        w = p[0];
        wp = p[1];
    }
};

// residues of three and four 64-bit words (wide.cuh); a twiddle entry is (w, w') of 2 NL words
template <int NL>
struct TraitsWide {
    typedef Wide<NL> E;
    typedef Wide<NL> TW;  // first of the entry's two values; the companion follows it
    static constexpr int EPR = 4;  // swizzle group (a permutation of each run of 4 residues)
    __device__ __forceinline__ static E make(const uint64_t *v) { return wide_from<NL>(v); }
    __device__ __forceinline__ static void load_tw(const TW *t, unsigned idx, E &w, E &wp) {
        const uint64_t *p = reinterpret_cast<const uint64_t *>(t) + 2 * NL * (size_t)idx;
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            w.w[k] = __ldg(reinterpret_cast<const unsigned long long *>(p) + k);
            wp.w[k] = __ldg(reinterpret_cast<const unsigned long long *>(p) + NL + k);
        }
    }
};
template <>
struct Traits<3> : TraitsWide<3> {};
template <>
struct Traits<4> : TraitsWide<4> {};

constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v >> 1); }
constexpr int maxc(int a, int b) { return a > b ? a : b; }

// Static shape of the kernel for tiles of 2^L residues.  RL = 0: the throughput shape (8 residues per
// thread, 4 for wide residues, several tiles per CTA of 256 threads).  RL > 0: the latency shape of
// launches with too few tiles to fill the GPU: RL residues per thread and one tile per CTA, so that
// a tile's butterflies spread over more warps and its CTAs over more SMs.
template <int W, int L, int RL = 0>
struct Shape {
    static constexpr int T = 1 << L;                 // residues per tile
    static constexpr int RMAX = RL ? RL : (W <= 2 ? 8 : 4);  // radix: wide residues hold 4 per thread
    static constexpr int R = T < RMAX ? T : RMAX;    // residues per thread (radix)
    static constexpr int r = ilog2c(R);              // stages per register round
    static constexpr int TPT = T / R;                // threads per tile
    // tiles per CTA: 256 threads for tiles up to 2^11 (up to 2^10 for wide residues), 512 for 2^12
    static constexpr int G = RL ? 1 : ((TPT <= 256) ? (256 / TPT) : 1);
    static constexpr int NT = G * TPT;               // threads per CTA
    static constexpr int TS = T + 1;                 // padded tile stride in shared memory
    static constexpr int ROUNDS = (L + r - 1) / r;
    static constexpr size_t SMEM = (size_t)G * TS * sizeof(typename Traits<W>::E);
    // the latency shape stages its tile's T - 1 twiddles in shared memory (entry 2^s + i: stage s)
    static constexpr size_t TWSMEM = RL ? (size_t)T * sizeof(typename Traits<W>::TW) : 0;
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

__device__ __forceinline__ uint64_t ld_cg(const uint64_t *p) { return __ldcg((const unsigned long long *)p); }
__device__ __forceinline__ uint4 ld_cg(const uint4 *p) { return __ldcg(p); }
__device__ __forceinline__ void st_cg(uint64_t *p, uint64_t v) { __stcg((unsigned long long *)p, (unsigned long long)v); }
__device__ __forceinline__ void st_cg(uint4 *p, uint4 v) { __stcg(p, v); }

// Barrier among the NT threads that run the tile code: the whole CTA (id 0) or, in a kernel
// with a separate producer warp, the named barrier BAR of the NT compute threads.
template <int BAR, int NT>
__device__ __forceinline__ void tile_sync() {
    if (BAR == 0)
        __syncthreads();
    else
        asm volatile("bar.sync %0, %1;" ::"n"(BAR), "n"(NT) : "memory");
}

// Per-tile addressing of one pass: for tile g of a CTA's group, the polynomial and the tile's
// index inside it (tiles per polynomial are a power of two).
struct TileAddr {
    int lgTP;
    unsigned long long mask;
    __device__ __forceinline__ TileAddr(const PassArgs &a) {
        lgTP = a.col ? (a.logN - a.L1) : a.L1;
        mask = (1ull << lgTP) - 1;
    }
};

// Stage tiles first_tile .. first_tile + G - 1 into `sm` with ordinary loads through L2.
template <int W, int L, int NTH = Shape<W, L>::NT, int RL = 0>
__device__ __forceinline__ void load_tiles_sync(const PassArgs &a, unsigned long long first_tile,
                                                typename Traits<W>::E *sm, int tid) {
    typedef typename Traits<W>::E E;
    typedef Shape<W, L, RL> S;
    const TileAddr ta(a);
    const E *in = reinterpret_cast<const E *>(a.in);
    const bool gfast = a.in_layout != LAYOUT_ROW;
    constexpr int PER = (S::G * S::T) / NTH;       // residues per thread
    constexpr int BATCH = PER < 16 ? PER : 16;      // loads in flight per thread
    static_assert(PER % BATCH == 0, "tile residues must split evenly");
#pragma unroll 1
    for (int c = 0; c < PER; c += BATCH) {
        E v[BATCH];
#pragma unroll
        for (int u = 0; u < BATCH; ++u) {
            const int i = tid + (c + u) * NTH;
            int g = gfast ? (i % S::G) : (i / S::T);
            int l = gfast ? (i / S::G) : (i % S::T);
            unsigned long long gt = first_tile + g;
            unsigned long long poly = gt >> ta.lgTP;
            unsigned ti = (unsigned)(gt & ta.mask);
            v[u] = poly < a.batch ? ld_cg(in + poly * a.in_stride + tile_pos(a.in_layout, ti, l, L, a.L1, a.logN, a.perm))
                                  : E();
        }
#pragma unroll
        for (int u = 0; u < BATCH; ++u) {
            const int i = tid + (c + u) * NTH;
            int g = gfast ? (i % S::G) : (i / S::T);
            int l = gfast ? (i / S::G) : (i % S::T);
            sm[g * S::TS + swz<W>(l)] = v[u];
        }
    }
}

__device__ __forceinline__ void cp_async(void *dst, const uint4 *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async(void *dst, const uint64_t *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// The same staging with asynchronous copies (cp.async): the caller commits the group and waits
// for it before the tiles are used.  Tiles past the last polynomial are left unfilled (their
// results are never stored).
template <int W, int L, int NTH = Shape<W, L>::NT, int RL = 0>
__device__ __forceinline__ void load_tiles_async(const PassArgs &a, unsigned long long first_tile,
                                                 typename Traits<W>::E *sm, int tid) {
    typedef typename Traits<W>::E E;
    typedef Shape<W, L, RL> S;
    const TileAddr ta(a);
    const E *in = reinterpret_cast<const E *>(a.in);
    const bool gfast = a.in_layout != LAYOUT_ROW;
    for (int i = tid; i < S::G * S::T; i += NTH) {
        int g = gfast ? (i % S::G) : (i / S::T);
        int l = gfast ? (i / S::G) : (i % S::T);
        unsigned long long gt = first_tile + g;
        unsigned long long poly = gt >> ta.lgTP;
        unsigned ti = (unsigned)(gt & ta.mask);
        if (poly < a.batch)
            cp_async(sm + g * S::TS + swz<W>(l), in + poly * a.in_stride + tile_pos(a.in_layout, ti, l, L, a.L1, a.logN, a.perm));
    }
}

// Twiddle base of a tile: stage s of the tile uses entries (base << s) + i, i < 2^s, of the
// direction's table (column pass: 1; row pass: 2^L1 + the tile's row, bit-reversed when the pass
// permutes its rows).
__device__ __forceinline__ unsigned tile_tw_base(const PassArgs &a, unsigned long long tile) {
    const TileAddr ta(a);
    const unsigned ti = (unsigned)(tile & ta.mask);
    return a.col ? 1u : ((1u << a.L1) + (a.perm ? brv(ti, a.L1) : ti));
}

// Copy the T - 1 twiddles of one tile (cp.async) into `dst`, entry (base << s) + i to 2^s + i, so
// that the rounds read them from shared memory with base 1.  Entries are 16 (64-bit) or 32 bytes.
template <int W, int L>
__device__ __forceinline__ void stage_twiddles_async(const PassArgs &a, unsigned long long tile,
                                                     typename Traits<W>::TW *dst, int tid, int nth) {
    typedef typename Traits<W>::TW TW;
    constexpr int CH = sizeof(TW) / 16;  // 16-byte chunks per entry
    const unsigned base = tile_tw_base(a, tile);
    const uint4 *src = reinterpret_cast<const uint4 *>(a.tw);
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    for (int c = tid; c < ((1 << L) - 1) * CH; c += nth) {
        const unsigned k = 1u + (unsigned)(c / CH);  // local entry 1 .. T - 1
        const int s = 31 - __clz(k);
        const unsigned gidx = (base << s) + (k - (1u << s));
        cp_async(d + k * CH + c % CH, src + (size_t)gidx * CH + c % CH);
    }
}

// Shared-memory index of element l of a tile: the tile's own swizzled array, or (XCOL) element l
// of tile gx in a column-view TMA group of 8 tiles, [l][gx ^ (l & 7)] (tma.cuh).
template <int W, bool XCOL>
__device__ __forceinline__ int tile_index(int l, int gx) {
    return XCOL ? ((l << 3) | (gx ^ (l & 7))) : swz<W>(l);
}

// One register round: stages s_begin .. s_begin + RR - 1 of a tile of 2^L residues, each thread
// holding R residues (R / 2^RR independent groups of 2^RR), read from and written back to the
// shared-memory tile, then a barrier (of the warp when one warp holds the tile).  s_begin is a runtime value so that all full rounds share
// this code (the instruction footprint matters when several kernels' tiles share one SM).
// XCOL: the tile is tile gx of a column-view TMA group, whose threads span the CTA's warps (the
// round ends with a CTA barrier); CANON: the last round of a final pass, which leaves canonical
// residues (below q) in shared memory for the copy engine to store.
template <int W, int L, int RR, bool INV, int BAR = 0, int RL = 0, bool XCOL = false, bool CANON = false>
__device__ __forceinline__ void radix_round(const PassArgs &a, typename Traits<W>::E *tile, int t, unsigned tw_base,
                                            int s_begin, const typename Traits<W>::TW *tw, typename Traits<W>::E q,
                                            typename Traits<W>::E q8, typename Traits<W>::E nq, int gx = 0) {
    typedef Traits<W> Tr;
    typedef typename Tr::E E;
    typedef Shape<W, L, RL> S;
    constexpr int V = S::R >> RR;  // independent groups per thread
    const int b_lo = L - s_begin - RR, b_hi = L - 1 - s_begin;
    E x[S::R];
    int base[V];
#pragma unroll
    for (int k = 0; k < V; ++k) {
        int vt = t + k * S::TPT;
        int lo = vt & ((1 << b_lo) - 1), hi = vt >> b_lo;
        base[k] = (hi << (b_hi + 1)) | lo;
#pragma unroll
        for (int e = 0; e < (1 << RR); ++e) x[k * (1 << RR) + e] = tile[tile_index<W, XCOL>(base[k] | (e << b_lo), gx)];
    }
#pragma unroll
    for (int jj = 0; jj < RR; ++jj) {
        const int j = INV ? (RR - 1 - jj) : jj;
        const int s = s_begin + j;           // local stage
        const int half = 1 << (RR - 1 - j);  // distance in the register index
#pragma unroll
        for (int k = 0; k < V; ++k) {
            // twiddle index of butterfly (k, e0): (tw_base << s) + (l0 >> (L - s)) with
            // l0 = base[k] | (e0 << b_lo); base[k] is zero in bits b_lo .. b_lo + RR - 1, so this is
            // tb + (e0 >> (RR - j)), a compile-time offset: butterflies that share a twiddle share
            // its load
            const unsigned tb = (tw_base << s) + ((unsigned)base[k] >> (L - s));
#pragma unroll
            for (int e0 = 0; e0 < (1 << RR); ++e0) {
                if (e0 & half) continue;
                const unsigned idx = tb + (unsigned)(e0 >> (RR - j));
                E &u = x[k * (1 << RR) + e0];
                E &v = x[k * (1 << RR) + e0 + half];
                E w, wp;
                if (!INV) {
                    if constexpr (RL > 0) Tr::load_tw_shared(tw, idx, w, wp);
                    else Tr::load_tw(tw, idx, w, wp);
                    E uu = csub(u, q8);                              // [0, 8q)
                    E tv = mul_mod_shoup_lazy(v, w, wp, q, nq);      // [0, 6q)
                    u = add_nored(uu, tv);                           // [0, 14q)
                    v = add_sub(uu, q8, tv);                         // (2q, 16q)
                } else if (s == 0 && a.scale) {
                    E dif = add_sub(u, q8, v);                       // (0, 16q)
                    E sum = add_nored(u, v);                         // [0, 16q)
                    u = mul_mod_shoup_lazy(sum, Tr::make(a.sc), Tr::make(a.scp), q, nq);
                    v = mul_mod_shoup_lazy(dif, Tr::make(a.ws), Tr::make(a.wsp), q, nq);
                } else {
                    if constexpr (RL > 0) Tr::load_tw_shared(tw, idx, w, wp);
                    else Tr::load_tw(tw, idx, w, wp);
                    E dif = add_sub(u, q8, v);                       // (0, 16q)
                    u = csub(add_nored(u, v), q8);                   // [0, 8q)
                    v = mul_mod_shoup_lazy(dif, w, wp, q, nq);       // [0, 6q)
                }
            }
        }
    }
    if constexpr (CANON) {  // forward values are below 16q, inverse ones below 8q
        const E q2 = add_nored(q, q), q4 = add_nored(q2, q2);
#pragma unroll
        for (int i = 0; i < S::R; ++i) {
            E v = x[i];
            if (!INV) v = csub(v, q8);
            v = csub(v, q4);
            v = csub(v, q2);
            x[i] = csub(v, q);
        }
    }
#pragma unroll
    for (int k = 0; k < V; ++k) {
#pragma unroll
        for (int e = 0; e < (1 << RR); ++e) tile[tile_index<W, XCOL>(base[k] | (e << b_lo), gx)] = x[k * (1 << RR) + e];
    }
    // A tile's TPT threads are consecutive: when they fit in one warp the next round reads only
    // what this warp wrote, and a warp barrier (which orders shared memory among its threads)
    // suffices; the warps of a CTA then drift apart between rounds instead of waiting for each other.
    if (S::TPT <= 32 && !XCOL)
        __syncwarp();
    else
        tile_sync<BAR, S::NT>();
}

// The register rounds of one pass on the CTA's staged tiles: every full round (three stages) runs
// the same code in a loop; a shorter round, when L is not a multiple of 3, has its own (forward:
// last, inverse: first).  Called by NT = Shape::NT threads; ends with a barrier of the NT threads.
template <int W, int L, bool INV, int BAR = 0, int RL = 0>
__device__ __forceinline__ void tile_rounds(const PassArgs &a, unsigned long long first_tile,
                                            typename Traits<W>::E *sm, int tid,
                                            const typename Traits<W>::TW *tw_sm = nullptr) {
    typedef Traits<W> Tr;
    typedef typename Tr::E E;
    typedef Shape<W, L, RL> S;
    const E q = Tr::make(a.q);
    const E q2 = add_nored(q, q), q4 = add_nored(q2, q2);
    const E q8 = add_nored(q4, q4);
    const E nq = neg(q);
    const int g = tid / S::TPT, t = tid % S::TPT;
    // the latency shape reads its tile's twiddles from the shared-memory copy, whose base is 1
    const typename Tr::TW *tw = RL ? tw_sm : reinterpret_cast<const typename Tr::TW *>(a.tw);
    const unsigned tw_base = RL ? 1u : tile_tw_base(a, first_tile + g);
    E *tile = sm + g * S::TS;
    constexpr int FULL = L / S::r, PART = L - FULL * S::r;
    if (!INV) {
#pragma unroll 1
        for (int rho = 0; rho < FULL; ++rho) radix_round<W, L, S::r, false, BAR, RL>(a, tile, t, tw_base, rho * S::r, tw, q, q8, nq);
        if (PART) radix_round<W, L, PART, false, BAR, RL>(a, tile, t, tw_base, FULL * S::r, tw, q, q8, nq);
    } else {
        if (PART) radix_round<W, L, PART, true, BAR, RL>(a, tile, t, tw_base, FULL * S::r, tw, q, q8, nq);
#pragma unroll 1
        for (int rho = FULL - 1; rho >= 0; --rho) radix_round<W, L, S::r, true, BAR, RL>(a, tile, t, tw_base, rho * S::r, tw, q, q8, nq);
    }
    if (S::TPT <= 32) tile_sync<BAR, S::NT>();  // what follows reads across tiles
}

// One CTA's share of a pass on tiles already staged in `sm` (by load_tiles_*): tiles
// first_tile .. first_tile + G - 1 of the batch, a tile past the last polynomial being skipped.
// Called by NT = Shape::NT threads with thread index tid after a barrier that follows the staging;
// ends with a barrier, after which `sm` may be refilled.
//
// Butterflies are lazy (after Harvey): between stages the values stay below 16q (forward) or 8q
// (inverse), and twiddle products are left below 6q (Shoup without its final correction: [0, 6q)
// at 128 bits, whose quotient comes from a truncated high product, [0, 2q) at 64 bits); the pass
// flagged `final` canonicalises what it stores.  q < 2^124 (2^60) keeps 16q below the word size.
//   forward (CT):  u <- u mod 8q;  t = w v mod q + {0, .., 5q};  (u, v) <- (u + t, u + 8q - t)
//   inverse (GS):  (u, v) <- ((u + v) mod 8q, (u + 8q - v) w mod q + {0, .., 5q})
// Global loads and stores go through L2 only (.cg), so a pass may read what another SM wrote
// earlier in the same kernel once the writer's completion is observed.
template <int W, int L, bool INV, int BAR = 0, int RL = 0>
__device__ __forceinline__ void tile_compute_store(const PassArgs &a, unsigned long long first_tile,
                                           typename Traits<W>::E *sm, int tid,
                                           const typename Traits<W>::TW *tw_sm = nullptr) {
    typedef Traits<W> Tr;
    typedef typename Tr::E E;
    typedef Shape<W, L, RL> S;

    const E q = Tr::make(a.q);
    const E q2 = add_nored(q, q);
    const E q4 = add_nored(q2, q2);
    const E q8 = add_nored(q4, q4);
    const int L1 = a.L1, logN = a.logN;
    const TileAddr ta(a);
    const int lgTP = ta.lgTP;
    const unsigned long long tp_mask = ta.mask;
    E *out = reinterpret_cast<E *>(a.out);
    const bool gfast_out = a.out_layout != LAYOUT_ROW;

    tile_rounds<W, L, INV, BAR, RL>(a, first_tile, sm, tid, tw_sm);

    // ---- shared -> global (canonical residues from the last pass)
    for (int i = tid; i < S::G * S::T; i += S::NT) {
        int gg = gfast_out ? (i % S::G) : (i / S::T);
        int l = gfast_out ? (i / S::G) : (i % S::T);
        unsigned long long gt = first_tile + gg;
        unsigned long long poly = gt >> lgTP;
        unsigned ti = (unsigned)(gt & tp_mask);
        if (poly < a.batch) {
            E v = sm[gg * S::TS + swz<W>(l)];
            if (a.final) {
                if (!INV) v = csub(v, q8);  // forward values are below 16q, inverse ones below 8q
                v = csub(v, q4);
                v = csub(v, q2);
                v = csub(v, q);
            }
            st_cg(out + poly * a.out_stride + tile_pos(a.out_layout, ti, l, L, L1, logN, a.perm), v);
        }
    }
    tile_sync<BAR, S::NT>();
}

// The whole pass for one CTA group with synchronous staging (used by the batched kernel).
template <int W, int L, bool INV>
__device__ __forceinline__ void tile_group(const PassArgs &a, unsigned long long first_tile,
                                           typename Traits<W>::E *sm, int tid) {
    load_tiles_sync<W, L>(a, first_tile, sm, tid);
    __syncthreads();
    tile_compute_store<W, L, INV>(a, first_tile, sm, tid);
}

// A pass over `groups` CTA groups by a persistent grid: each CTA walks the groups with a stride
// of gridDim.x and prefetches the next group's tiles (cp.async into the second of two shared
// buffers) while it transforms the current one.  RL > 0 selects the latency shape (one tile per
// CTA), whose registers are capped so that 1024 threads fit an SM.
template <int W, int L, int RL>
constexpr int pass_min_blocks() {
    return RL ? (1024 / Shape<W, L, RL>::NT < 32 ? 1024 / Shape<W, L, RL>::NT : 32)
              : (W > 2 ? 2 : ((Shape<W, L>::NT <= 256) ? (W == 1 ? 4 : 3) : 1));
}

template <int W, int L, bool INV, int RL = 0>
__global__ void __launch_bounds__(Shape<W, L, RL>::NT, (pass_min_blocks<W, L, RL>()))
    ntt_pass_kernel(const PassArgs a, unsigned long long groups) {
    typedef typename Traits<W>::E E;
    typedef typename Traits<W>::TW TW;
    typedef Shape<W, L, RL> S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // [twiddles 0][twiddles 1] (latency shape only; 16-byte entries or pairs) [tiles 0][tiles 1]
    TW *tws0 = reinterpret_cast<TW *>(smem_raw), *tws1 = tws0 + (RL ? S::T : 0);
    E *buf0 = reinterpret_cast<E *>(smem_raw + 2 * S::TWSMEM), *buf1 = buf0 + S::G * S::TS;
    const int tid = threadIdx.x;
    unsigned long long grp = blockIdx.x;
    if (grp < groups) {
        load_tiles_async<W, L, S::NT, RL>(a, grp * S::G, buf0, tid);
        if constexpr (RL > 0) stage_twiddles_async<W, L>(a, grp, tws0, tid, S::NT);
    }
    cp_async_commit();
    bool odd = false;
    for (; grp < groups; grp += gridDim.x) {
        E *cur = odd ? buf1 : buf0, *nxt = odd ? buf0 : buf1;
        TW *twc = odd ? tws1 : tws0, *twn = odd ? tws0 : tws1;
        const unsigned long long next = grp + gridDim.x;
        if (next < groups) {
            load_tiles_async<W, L, S::NT, RL>(a, next * S::G, nxt, tid);
            if constexpr (RL > 0) stage_twiddles_async<W, L>(a, next, twn, tid, S::NT);
        }
        cp_async_commit();
        cp_async_wait_1();  // this thread's copies of the current group have landed
        __syncthreads();    // and everyone else's
        tile_compute_store<W, L, INV, 0, RL>(a, grp * S::G, cur, tid, twc);
        odd = !odd;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

__host__ __forceinline__ int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

__host__ __forceinline__ unsigned long long pass_tiles(const PassArgs &a) {
    const unsigned long long TP = a.col ? (1ull << (a.logN - a.L1)) : (1ull << a.L1);
    return TP * a.batch;
}

template <int W, int L, bool INV, int RL = 0>
cudaError_t launch_one(const PassArgs &a, cudaStream_t s) {
    typedef Shape<W, L, RL> S;
    static int per_sm = 0;  // benign race: every thread computes the same values
    const size_t smem = 2 * S::SMEM + 2 * S::TWSMEM;
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(ntt_pass_kernel<W, L, INV, RL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, ntt_pass_kernel<W, L, INV, RL>, S::NT, smem);
        if (e != cudaSuccess) return e;
        per_sm = n > 0 ? n : 1;
    }
    const unsigned long long groups = (pass_tiles(a) + S::G - 1) / S::G;
    if (groups == 0) return cudaSuccess;
    const unsigned long long wave = (unsigned long long)sm_count() * per_sm;
    const unsigned grid = (unsigned)(groups < wave ? groups : wave);
    ntt_pass_kernel<W, L, INV, RL><<<grid, S::NT, smem, s>>>(a, groups);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// The TMA form of the throughput pass (128-bit residues, tiles of 2^8): each CTA group of 8 tiles
// arrives as one tensor copy into a 1024-byte aligned buffer and leaves as one (tma.cuh), so the
// threads only transform.  Column view: the group lands as [l][c ^ (l & 7)]; thread (g, t) =
// (tid & 7, tid >> 3) works on tile g, so that each quarter-warp touches the 8 tiles at one
// element, conflict-free, and rounds end with a CTA barrier (a tile's threads span the warps).
// Row view: the group lands as 8 swizzled tiles, each held by one warp as in the cp.async form.
// The last round of a final pass leaves canonical residues for the store.
// ------------------------------------------------------------------------------------------------

constexpr unsigned TMA_GROUP_BYTES = Shape<2, TMA_L>::G * Shape<2, TMA_L>::T * 16;  // 32 KiB
constexpr size_t TMA_SMEM = 2 * (size_t)TMA_GROUP_BYTES + 1024;                      // + alignment
constexpr unsigned long long TMA_WAIT_NS = 1000000000ull;  // bound of a copy wait (never reached)

// Fault word of the TMA pass (one per translation unit): the group index + 1 of a copy wait that
// gave up, after which the kernel stops.  Not expected to be set: a tensor copy of an in-bounds
// box always completes; the bound only keeps a broken copy from hanging the GPU.
static __device__ unsigned long long g_tma_fault;

// Box coordinates (x words, y rows, polynomial) of the group of 8 tiles that starts at tile gt
__device__ __forceinline__ void tma_box(const TileAddr &ta, bool col, unsigned long long gt, int &x, int &y, int &z) {
    constexpr int T = Shape<2, TMA_L>::T;
    const unsigned ti = (unsigned)(gt & ta.mask);
    z = (int)(gt >> ta.lgTP);
    x = col ? (int)(2 * ti) : 0;
    y = col ? 0 : (int)(ti * (T / 8));
}

template <bool INV, bool COL>
__device__ __forceinline__ void tma_rounds(const PassArgs &a, uint4 *buf, unsigned long long gt0, int tid) {
    typedef Traits<2> Tr;
    typedef Tr::E E;
    typedef Shape<2, TMA_L> S;
    constexpr int L = TMA_L, r = S::r, FULL = L / r, PART = L - FULL * r;
    static_assert(PART > 0 && S::TPT == 32 && S::G == 8, "the TMA form's round schedule is that of tiles of 2^8");
    const E q = Tr::make(a.q);
    const E q2 = add_nored(q, q), q4 = add_nored(q2, q2);
    const E q8 = add_nored(q4, q4);
    const E nq = neg(q);
    const Tw128 *tw = reinterpret_cast<const Tw128 *>(a.tw);
    const int g = COL ? (tid & 7) : (tid >> 5), t = COL ? (tid >> 3) : (tid & 31);
    E *tile = COL ? buf : buf + g * S::T;
    const unsigned tw_base = COL ? 1u : tile_tw_base(a, gt0 + g);
    if (!INV) {
#pragma unroll 1
        for (int rho = 0; rho < FULL; ++rho)
            radix_round<2, L, r, false, 0, 0, COL, false>(a, tile, t, tw_base, rho * r, tw, q, q8, nq, g);
        if (a.final) radix_round<2, L, PART, false, 0, 0, COL, true>(a, tile, t, tw_base, FULL * r, tw, q, q8, nq, g);
        else radix_round<2, L, PART, false, 0, 0, COL, false>(a, tile, t, tw_base, FULL * r, tw, q, q8, nq, g);
    } else {
        radix_round<2, L, PART, true, 0, 0, COL, false>(a, tile, t, tw_base, FULL * r, tw, q, q8, nq, g);
#pragma unroll 1
        for (int rho = FULL - 1; rho >= 1; --rho)
            radix_round<2, L, r, true, 0, 0, COL, false>(a, tile, t, tw_base, rho * r, tw, q, q8, nq, g);
        if (a.final) radix_round<2, L, r, true, 0, 0, COL, true>(a, tile, t, tw_base, 0, tw, q, q8, nq, g);
        else radix_round<2, L, r, true, 0, 0, COL, false>(a, tile, t, tw_base, 0, tw, q, q8, nq, g);
    }
}

// A pass over `groups` groups by a persistent grid, double-buffered: thread 0 issues the next
// group's tensor copy while the CTA transforms the current one, and the store of each group.
template <bool INV, bool COL>
__global__ void __launch_bounds__(256, 3)
    ntt_pass_tma_kernel(const __grid_constant__ CUtensorMap tm_in, const __grid_constant__ CUtensorMap tm_out,
                        const PassArgs a, unsigned long long groups) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_ok;
    const int tid = threadIdx.x;
    unsigned char *p = smem_raw + ((1024u - (tma::su32(smem_raw) & 1023u)) & 1023u);
    uint4 *const buf0 = reinterpret_cast<uint4 *>(p), *const buf1 = reinterpret_cast<uint4 *>(p + TMA_GROUP_BYTES);
    const TileAddr ta(a);
    unsigned long long grp = blockIdx.x;
    if (tid == 0) {
        tma::mbar_init(&bar[0], 1);
        tma::mbar_init(&bar[1], 1);
        tma::mbar_init_fence();
        tma::prefetch_map(&tm_in);
        tma::prefetch_map(&tm_out);
        if (grp < groups) {
            int x, y, z;
            tma_box(ta, COL, grp * Shape<2, TMA_L>::G, x, y, z);
            tma::mbar_expect(&bar[0], TMA_GROUP_BYTES);
            tma::load3(buf0, &tm_in, x, y, z, &bar[0]);
        }
    }
    __syncthreads();
    unsigned ph0 = 0, ph1 = 0;
    bool odd = false;
    for (; grp < groups; grp += gridDim.x, odd = !odd) {
        uint4 *cur = odd ? buf1 : buf0, *nxt = odd ? buf0 : buf1;
        uint64_t *bc = odd ? &bar[1] : &bar[0], *bn = odd ? &bar[0] : &bar[1];
        const unsigned ph = odd ? ph1 : ph0;
        const unsigned long long next = grp + gridDim.x;
        if (tid == 0) {
            if (next < groups) {
                tma::store_wait_read();  // the other buffer's store has read it
                int x, y, z;
                tma_box(ta, COL, next * Shape<2, TMA_L>::G, x, y, z);
                tma::mbar_expect(bn, TMA_GROUP_BYTES);
                tma::load3(nxt, &tm_in, x, y, z, bn);
            }
            s_ok = tma::mbar_wait(bc, ph, TMA_WAIT_NS);
        }
        __syncthreads();
        if (!s_ok) {
            if (tid == 0) {  // record the fault, then wait (bounded again) for the copies in flight
                atomicCAS(&g_tma_fault, 0ull, grp + 1);
                tma::mbar_wait(bc, ph, TMA_WAIT_NS);
                if (next < groups) tma::mbar_wait(bn, odd ? ph0 : ph1, TMA_WAIT_NS);
            }
            break;
        }
        while (!tma::mbar_test(bc, ph)) {  // completed: thread 0 saw it
        }
        if (odd) ph1 ^= 1;
        else ph0 ^= 1;
        tma_rounds<INV, COL>(a, cur, grp * Shape<2, TMA_L>::G, tid);
        tma::fence_async_shared();
        __syncthreads();
        if (tid == 0) {
            int x, y, z;
            tma_box(ta, COL, grp * Shape<2, TMA_L>::G, x, y, z);
            tma::store3(&tm_out, x, y, z, cur);
            tma::store_commit();
        }
    }
    if (tid == 0) tma::store_wait();
}

template <bool INV>
cudaError_t launch_tma(const PassArgs &a, cudaStream_t s, bool *taken) {
    *taken = false;
    if (!tma_eligible(a)) return cudaSuccess;
    const unsigned long long groups = pass_tiles(a) / Shape<2, TMA_L>::G;
    if (groups < (unsigned long long)sm_count()) return cudaSuccess;  // small passes: the latency shape
    CUtensorMap mi, mo;
    if (tile_map(&mi, a.col != 0, a.in, a.logN, a.L1, a.batch, a.in_stride) ||
        tile_map(&mo, a.col != 0, a.out, a.logN, a.L1, a.batch, a.out_stride))
        return cudaSuccess;
    static int per_sm[2] = {0, 0};  // benign race: every thread computes the same values
    const int c = a.col ? 1 : 0;
    if (per_sm[c] == 0) {
        auto k = a.col ? ntt_pass_tma_kernel<INV, true> : ntt_pass_tma_kernel<INV, false>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TMA_SMEM);
        if (e != cudaSuccess) return e;
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, 256, TMA_SMEM);
        if (e != cudaSuccess) return e;
        per_sm[c] = n > 0 ? n : 1;
    }
    const unsigned long long wave = (unsigned long long)sm_count() * per_sm[c];
    const unsigned grid = (unsigned)(groups < wave ? groups : wave);
    if (a.col) ntt_pass_tma_kernel<INV, true><<<grid, 256, TMA_SMEM, s>>>(mi, mo, a, groups);
    else ntt_pass_tma_kernel<INV, false><<<grid, 256, TMA_SMEM, s>>>(mi, mo, a, groups);
    *taken = true;
    return cudaGetLastError();
}

// Residues per thread of the latency shape: radix-4 rounds.  Measured on a single transform of
// 2^10 (124-bit, forward + inverse): 13.6 us with radix-2 rounds, 12.1 with radix-4, 16.1 with
// radix-8 (fewer warps per tile).
constexpr int LATENCY_RADIX = 4;

// One pass: the throughput shape, or the latency shape (radix-4 rounds, one tile of 2^L residues on
// 2^(L-2) threads, its twiddles staged in shared memory) when the throughput shape's CTAs would
// not give every SM one (a single polynomial or a small batch), for one- and two-word residues
// and tiles of 2^5 to 2^10 (larger tiles already take a CTA each in the throughput shape).
template <int W, int L, bool INV>
cudaError_t launch_pass(const PassArgs &a, cudaStream_t s) {
    if constexpr (W == 2 && L == TMA_L) {
        bool taken = false;
        cudaError_t e = launch_tma<INV>(a, s, &taken);
        if (e != cudaSuccess || taken) return e;
    }
    if constexpr (W <= 2 && L >= 5 && L <= 10) {
        const unsigned long long groups = (pass_tiles(a) + Shape<W, L>::G - 1) / Shape<W, L>::G;
        if (groups < (unsigned long long)sm_count()) return launch_one<W, L, INV, LATENCY_RADIX>(a, s);
    }
    return launch_one<W, L, INV>(a, s);
}

template <int W, bool INV>
cudaError_t launch_w(int L, const PassArgs &a, cudaStream_t s) {
    switch (L) {
    case 1: return launch_pass<W, 1, INV>(a, s);
    case 2: return launch_pass<W, 2, INV>(a, s);
    case 3: return launch_pass<W, 3, INV>(a, s);
    case 4: return launch_pass<W, 4, INV>(a, s);
    case 5: return launch_pass<W, 5, INV>(a, s);
    case 6: return launch_pass<W, 6, INV>(a, s);
    case 7: return launch_pass<W, 7, INV>(a, s);
    case 8: return launch_pass<W, 8, INV>(a, s);
    case 9: return launch_pass<W, 9, INV>(a, s);
    case 10: return launch_pass<W, 10, INV>(a, s);
    case 11: return launch_pass<W, 11, INV>(a, s);
    case 12: return launch_pass<W, 12, INV>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ntt_detail
}  // namespace mq

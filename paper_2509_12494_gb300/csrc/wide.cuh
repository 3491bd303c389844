// wide.cuh -- residues of three and four 64-bit words (192- and 256-bit integers; q < 2^188 or
// q < 2^252, so that 16q fits the word as the lazy butterflies need), the larger bit-widths that
// Sec. 7 names.  The same operations as residue.cuh, written over 64-bit limbs with 128-bit
// intermediate products and sums (the double-word products of Sec. 2.2, Eq. 8, one level up):
// simple and exact rather than tuned, for the widths beyond the paper's 128 bits.
#pragma once
#include <stdint.h>

namespace mq {

typedef unsigned __int128 u128d;

template <int NL>
struct __align__(NL == 4 ? 16 : 8) Wide {
    uint64_t w[NL];  // little-endian 64-bit limbs
};

template <int NL>
__device__ __forceinline__ Wide<NL> wide_from(const uint64_t *v) {
    Wide<NL> r;
#pragma unroll
    for (int k = 0; k < NL; ++k) r.w[k] = v[k];
    return r;
}

// a + b mod 2^(64 NL)
template <int NL>
__device__ __forceinline__ Wide<NL> add_nored(const Wide<NL> &a, const Wide<NL> &b) {
    Wide<NL> r;
    uint64_t c = 0;
#pragma unroll
    for (int k = 0; k < NL; ++k) {
        const u128d t = (u128d)a.w[k] + b.w[k] + c;
        r.w[k] = (uint64_t)t;
        c = (uint64_t)(t >> 64);
    }
    return r;
}

// a - b mod 2^(64 NL); borrow = 1 if a < b
template <int NL>
__device__ __forceinline__ Wide<NL> sub_wide(const Wide<NL> &a, const Wide<NL> &b, uint64_t &borrow) {
    Wide<NL> r;
    uint64_t br = 0;
#pragma unroll
    for (int k = 0; k < NL; ++k) {
        const u128d t = (u128d)a.w[k] - b.w[k] - br;
        r.w[k] = (uint64_t)t;
        br = (uint64_t)(t >> 64) & 1u;
    }
    borrow = br;
    return r;
}

template <int NL>
__device__ __forceinline__ Wide<NL> sub_wide(const Wide<NL> &a, const Wide<NL> &b) {
    uint64_t br;
    return sub_wide(a, b, br);
}

// a >= m ? a - m : a
template <int NL>
__device__ __forceinline__ Wide<NL> csub(const Wide<NL> &a, const Wide<NL> &m) {
    uint64_t br;
    const Wide<NL> d = sub_wide(a, m, br);
    Wide<NL> r;
#pragma unroll
    for (int k = 0; k < NL; ++k) r.w[k] = br ? a.w[k] : d.w[k];
    return r;
}

// a + b2 - c for values that keep the result in [0, 2^(64 NL)): c <= a + b2
template <int NL>
__device__ __forceinline__ Wide<NL> add_sub(const Wide<NL> &a, const Wide<NL> &b2, const Wide<NL> &c) {
    return sub_wide(add_nored(a, b2), c);
}

template <int NL>
__device__ __forceinline__ Wide<NL> neg(const Wide<NL> &q) {
    Wide<NL> z;
#pragma unroll
    for (int k = 0; k < NL; ++k) z.w[k] = 0;
    return sub_wide(z, q);
}

template <int NL>
__device__ __forceinline__ Wide<NL> add_mod(const Wide<NL> &a, const Wide<NL> &b, const Wide<NL> &q) {
    return csub(add_nored(a, b), q);
}

template <int NL>
__device__ __forceinline__ Wide<NL> sub_mod(const Wide<NL> &a, const Wide<NL> &b, const Wide<NL> &q) {
    uint64_t br;
    const Wide<NL> d = sub_wide(a, b, br);
    return br ? add_nored(d, q) : d;
}

// Full product a * b as 2 NL limbs (operand scanning: row i adds a * b_i at limb i).
template <int NL>
__device__ __forceinline__ void mul_full(const Wide<NL> &a, const Wide<NL> &b, uint64_t r[2 * NL]) {
#pragma unroll
    for (int k = 0; k < 2 * NL; ++k) r[k] = 0;
#pragma unroll
    for (int i = 0; i < NL; ++i) {
        uint64_t c = 0;
#pragma unroll
        for (int j = 0; j < NL; ++j) {
            const u128d t = (u128d)a.w[j] * b.w[i] + r[i + j] + c;
            r[i + j] = (uint64_t)t;
            c = (uint64_t)(t >> 64);
        }
        r[i + NL] = c;
    }
}

// floor((a * b - D) / 2^(64 NL)) where D is the sum of the limb products a_j b_i with
// i + j <= NL - 2, which reach limbs 0 .. NL - 1 only: D < (NL - 1) 2^(64 NL) (1 + 2^-63), so the
// result is the true high half minus at most NL.
template <int NL>
__device__ __forceinline__ Wide<NL> mul_hi_trunc(const Wide<NL> &a, const Wide<NL> &b) {
    uint64_t r[2 * NL];
#pragma unroll
    for (int k = 0; k < 2 * NL; ++k) r[k] = 0;
#pragma unroll
    for (int i = 0; i < NL; ++i) {
        uint64_t c = 0;
#pragma unroll
        for (int j = 0; j < NL; ++j) {
            if (i + j < NL - 1) continue;
            const u128d t = (u128d)a.w[j] * b.w[i] + r[i + j] + c;
            r[i + j] = (uint64_t)t;
            c = (uint64_t)(t >> 64);
        }
        r[i + NL] = c;
    }
    Wide<NL> h;
#pragma unroll
    for (int k = 0; k < NL; ++k) h.w[k] = r[NL + k];
    return h;
}

// low NL limbs of a * b + c * d
template <int NL>
__device__ __forceinline__ Wide<NL> mul_lo2(const Wide<NL> &a, const Wide<NL> &b, const Wide<NL> &c,
                                            const Wide<NL> &d) {
    uint64_t r[NL];
#pragma unroll
    for (int k = 0; k < NL; ++k) r[k] = 0;
#pragma unroll
    for (int i = 0; i < NL; ++i) {
        uint64_t ca = 0, cc = 0;
#pragma unroll
        for (int j = 0; i + j < NL; ++j) {
            const u128d t = (u128d)a.w[j] * b.w[i] + r[i + j] + ca;
            r[i + j] = (uint64_t)t;
            ca = (uint64_t)(t >> 64);
        }
#pragma unroll
        for (int j = 0; i + j < NL; ++j) {
            const u128d t = (u128d)c.w[j] * d.w[i] + r[i + j] + cc;
            r[i + j] = (uint64_t)t;
            cc = (uint64_t)(t >> 64);
        }
    }
    Wide<NL> s;
#pragma unroll
    for (int k = 0; k < NL; ++k) s.w[k] = r[k];
    return s;
}

// a * w mod q up to NL + 1 multiples of q (Shoup with w' = floor(w 2^(64 NL) / q), a truncated
// quotient and no correction): in [0, (NL + 2) q), below 6q for both widths.  nq = 2^(64 NL) - q.
template <int NL>
__device__ __forceinline__ Wide<NL> mul_mod_shoup_lazy(const Wide<NL> &a, const Wide<NL> &w, const Wide<NL> &wp,
                                                       const Wide<NL> &q, const Wide<NL> &nq) {
    (void)q;
    return mul_lo2(a, w, mul_hi_trunc(a, wp), nq);
}

// a * w mod q, canonical (the exact Shoup quotient, one correction)
template <int NL>
__device__ __forceinline__ Wide<NL> mul_mod_shoup(const Wide<NL> &a, const Wide<NL> &w, const Wide<NL> &wp,
                                                  const Wide<NL> &q) {
    uint64_t h[2 * NL];
    mul_full(a, wp, h);
    Wide<NL> qhat;
#pragma unroll
    for (int k = 0; k < NL; ++k) qhat.w[k] = h[NL + k];
    return csub(mul_lo2(a, w, qhat, neg(q)), q);
}

// floor(x / 2^s) of a 2 NL-limb x whose quotient fits NL limbs; s uniform across the warp
template <int NL>
__device__ __forceinline__ Wide<NL> shr_wide(const uint64_t x[2 * NL], int s) {
    const int o = s >> 6, b = s & 63;
    Wide<NL> r;
#pragma unroll
    for (int k = 0; k < NL; ++k) {
        uint64_t lo = 0, hi = 0;
#pragma unroll
        for (int t = 0; t < 2 * NL; ++t) {  // select x[o + k], x[o + k + 1] without dynamic indexing
            if (t == o + k) lo = x[t];
            if (t == o + k + 1) hi = x[t];
        }
        r.w[k] = b ? ((lo >> b) | (hi << (64 - b))) : lo;
    }
    return r;
}

template <int NL>
struct ModW {
    Wide<NL> q, mu;  // mu = floor(2^(2L) / q)
    int L;           // bit length of q
};

// a * b mod q for any a, b < q (Barrett, Sec. 2.1, Eq. 4): quotient estimate
// floor(floor(x / 2^(L-1)) mu / 2^(L+1)), at most 2 below the true quotient
template <int NL>
__device__ __forceinline__ Wide<NL> mul_mod_barrett(const Wide<NL> &a, const Wide<NL> &b, const ModW<NL> &m) {
    uint64_t x[2 * NL], t[2 * NL];
    mul_full(a, b, x);
    const Wide<NL> q1 = shr_wide<NL>(x, m.L - 1);
    mul_full(q1, m.mu, t);
    const Wide<NL> q3 = shr_wide<NL>(t, m.L + 1);
    Wide<NL> lo;
#pragma unroll
    for (int k = 0; k < NL; ++k) lo.w[k] = x[k];
    Wide<NL> z;
#pragma unroll
    for (int k = 0; k < NL; ++k) z.w[k] = 0;
    Wide<NL> r = mul_lo2(q3, m.q, z, z);   // q3 q mod 2^(64 NL)
    r = sub_wide(lo, r);                   // x - q3 q < 3q
    r = csub(r, m.q);
    return csub(r, m.q);
}

// global memory: loads and stores through L2 only, and asynchronous copies into shared memory
__device__ __forceinline__ Wide<3> ld_cg(const Wide<3> *p) {
    const unsigned long long *s = reinterpret_cast<const unsigned long long *>(p);
    Wide<3> r;
    r.w[0] = __ldcg(s);
    r.w[1] = __ldcg(s + 1);
    r.w[2] = __ldcg(s + 2);
    return r;
}
__device__ __forceinline__ Wide<4> ld_cg(const Wide<4> *p) {
    const uint4 *s = reinterpret_cast<const uint4 *>(p);
    const uint4 a = __ldcg(s), b = __ldcg(s + 1);
    Wide<4> r;
    r.w[0] = a.x | ((uint64_t)a.y << 32);
    r.w[1] = a.z | ((uint64_t)a.w << 32);
    r.w[2] = b.x | ((uint64_t)b.y << 32);
    r.w[3] = b.z | ((uint64_t)b.w << 32);
    return r;
}
__device__ __forceinline__ void st_cg(Wide<3> *p, const Wide<3> &v) {
    unsigned long long *d = reinterpret_cast<unsigned long long *>(p);
    __stcg(d, v.w[0]);
    __stcg(d + 1, v.w[1]);
    __stcg(d + 2, v.w[2]);
}
__device__ __forceinline__ void st_cg(Wide<4> *p, const Wide<4> &v) {
    uint4 *d = reinterpret_cast<uint4 *>(p);
    __stcg(d, make_uint4((uint32_t)v.w[0], (uint32_t)(v.w[0] >> 32), (uint32_t)v.w[1], (uint32_t)(v.w[1] >> 32)));
    __stcg(d + 1, make_uint4((uint32_t)v.w[2], (uint32_t)(v.w[2] >> 32), (uint32_t)v.w[3], (uint32_t)(v.w[3] >> 32)));
}
__device__ __forceinline__ void cp_async(void *dst, const Wide<3> *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const char *s = reinterpret_cast<const char *>(src);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(s) : "memory");
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d + 8), "l"(s + 8) : "memory");
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d + 16), "l"(s + 16) : "memory");
}
__device__ __forceinline__ void cp_async(void *dst, const Wide<4> *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const char *s = reinterpret_cast<const char *>(src);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(s) : "memory");
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + 16), "l"(s + 16) : "memory");
}

}  // namespace mq

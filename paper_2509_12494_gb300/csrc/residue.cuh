// residue.cuh -- modular arithmetic on 64-bit and 128-bit residues for sm_103a.
//
// 128-bit values are uint4 = four 32-bit limbs, x lowest (the memory image of a little-endian
// unsigned 128-bit integer, i.e. {lo word, hi word}).  Word operations follow the double-word
// arithmetic of Sec. 2.2: additions with carry and subtractions with borrow are PTX carry chains
// (add.cc/addc, sub.cc/subc -- the GPU's native form of the adc/sbb instructions that MQX adds to
// AVX-512, Table 2), and products use the widening multiply halves mul.lo/mul.hi fused into
// mad.lo.cc/madc.hi.cc chains (schoolbook, Eq. 5).
//
// Modular operations (Sec. 2.1):
//   add_mod / sub_mod   conditional correction (Eq. 2 and 3): one add (sub) chain, one trial
//                       subtraction (addition) of q, and a select on the borrow;
//   mul_mod_barrett     general operands, Barrett reduction (Eq. 4 of Sec. 2.1) with
//                       L = bitlen(q), mu = floor(2^(2L) / q), quotient estimate
//                       floor(floor(x / 2^(L-1)) * mu / 2^(L+1)), which is at most 2 below the
//                       true quotient, so at most two conditional subtractions follow;
//   mul_mod_shoup       a fixed multiplier w with companion w' = floor(w * 2^B / q) (B = 64 or 128):
//                       qhat = floor(a * w' / 2^B) is the true quotient or one less (Shoup's
//                       method), so one conditional subtraction follows.  Used for twiddles.
// Preconditions: q odd, q < 2^60 (64-bit residues) or q < 2^124 (128-bit residues, the bound of
// Sec. 2.1 for 128-bit words); operands canonical (< q).  Results are canonical.
#pragma once
#include <stdint.h>

namespace mq {

// ------------------------------------------------------------------------------------------------
// 64-bit residues
// ------------------------------------------------------------------------------------------------

struct Mod64 {
    uint64_t q;   // modulus, odd, < 2^60
    uint64_t mu;  // floor(2^(2L) / q)
    int L;        // bit length of q
};

__device__ __forceinline__ uint64_t add_mod(uint64_t a, uint64_t b, uint64_t q) {
    uint64_t s = a + b;  // < 2^61, no overflow
    uint64_t d = s - q;
    return (s >= q) ? d : s;
}

__device__ __forceinline__ uint64_t sub_mod(uint64_t a, uint64_t b, uint64_t q) {
    uint64_t d = a - b;
    return (a < b) ? d + q : d;
}

// a * w mod q with w' = floor(w * 2^64 / q), a < 2^64, w < q < 2^63.
__device__ __forceinline__ uint64_t mul_mod_shoup(uint64_t a, uint64_t w, uint64_t wp, uint64_t q) {
    uint64_t qhat = __umul64hi(a, wp);
    uint64_t r = a * w - qhat * q;  // exact: the true remainder plus 0 or q, < 2q < 2^64
    return (r >= q) ? r - q : r;
}

// a * w mod q up to one multiple of q: in [0, 2q) (the final Shoup correction skipped).
__device__ __forceinline__ uint64_t mul_mod_shoup_lazy(uint64_t a, uint64_t w, uint64_t wp, uint64_t q) {
    return a * w - __umul64hi(a, wp) * q;
}
__device__ __forceinline__ uint64_t csub(uint64_t a, uint64_t m) { return a >= m ? a - m : a; }
__device__ __forceinline__ uint64_t add_nored(uint64_t a, uint64_t b) { return a + b; }
__device__ __forceinline__ uint64_t add_sub(uint64_t a, uint64_t b2, uint64_t c) { return a + b2 - c; }

// a * b mod q for any a, b < q (Barrett, Sec. 2.1).
__device__ __forceinline__ uint64_t mul_mod_barrett(uint64_t a, uint64_t b, const Mod64 &m) {
    uint64_t xlo = a * b, xhi = __umul64hi(a, b);           // x = a*b < 2^(2L)
    int s1 = m.L - 1;                                         // 1 <= s1 <= 59
    uint64_t q1 = (xlo >> s1) | (xhi << (64 - s1));           // floor(x / 2^(L-1)) < 2^(L+1)
    uint64_t q2lo = q1 * m.mu, q2hi = __umul64hi(q1, m.mu);   // q1 * mu < 2^(2L+2)
    int s3 = m.L + 1;                                         // 3 <= s3 <= 61
    uint64_t q3 = (q2lo >> s3) | (q2hi << (64 - s3));         // floor(q1 * mu / 2^(L+1))
    uint64_t r = xlo - q3 * m.q;                              // < 3q < 2^62, exact mod 2^64
    r = (r >= m.q) ? r - m.q : r;
    r = (r >= m.q) ? r - m.q : r;
    return r;
}

// ------------------------------------------------------------------------------------------------
// 128-bit residues (uint4 limbs, x lowest)
// ------------------------------------------------------------------------------------------------

struct Mod128 {
    uint4 q;   // modulus, odd, < 2^124
    uint4 mu;  // floor(2^(2L) / q) < 2^(L+1)
    int L;     // bit length of q
};

__device__ __forceinline__ uint4 add128(uint4 a, uint4 b) {
    uint4 r;
    asm("add.cc.u32  %0, %4, %8;\n\t"
        "addc.cc.u32 %1, %5, %9;\n\t"
        "addc.cc.u32 %2, %6, %10;\n\t"
        "addc.u32    %3, %7, %11;"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y), "r"(b.z), "r"(b.w));
    return r;
}

// r = a - b mod 2^128; mask = 0xffffffff if a < b (a borrow left the chain), else 0.
__device__ __forceinline__ uint4 sub128(uint4 a, uint4 b, uint32_t &mask) {
    uint4 r;
    asm("sub.cc.u32  %0, %5, %9;\n\t"
        "subc.cc.u32 %1, %6, %10;\n\t"
        "subc.cc.u32 %2, %7, %11;\n\t"
        "subc.cc.u32 %3, %8, %12;\n\t"
        "subc.u32    %4, 0, 0;"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w), "=r"(mask)
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y), "r"(b.z), "r"(b.w));
    return r;
}

__device__ __forceinline__ uint4 sel128(uint32_t mask, uint4 if_set, uint4 if_clear) {
    return make_uint4((if_set.x & mask) | (if_clear.x & ~mask), (if_set.y & mask) | (if_clear.y & ~mask),
                      (if_set.z & mask) | (if_clear.z & ~mask), (if_set.w & mask) | (if_clear.w & ~mask));
}

__device__ __forceinline__ uint4 and128(uint4 a, uint32_t mask) {
    return make_uint4(a.x & mask, a.y & mask, a.z & mask, a.w & mask);
}

// r < 2q  ->  r mod q
__device__ __forceinline__ uint4 reduce_once(uint4 r, uint4 q) {
    uint32_t m;
    uint4 d = sub128(r, q, m);
    return sel128(m, r, d);
}

__device__ __forceinline__ uint4 add_mod(uint4 a, uint4 b, uint4 q) {
    return reduce_once(add128(a, b), q);  // a + b < 2q < 2^125
}

__device__ __forceinline__ uint4 sub_mod(uint4 a, uint4 b, uint4 q) {
    uint32_t m;
    uint4 d = sub128(a, b, m);
    return add128(d, and128(q, m));  // add q back only when a < b
}

// 32 x 32 -> 64-bit product as (lo, hi): one full-rate wide multiply (a separate high-half multiply
// issues at half the rate of a low-half one on this GPU).
__device__ __forceinline__ void mul_wide32(uint32_t a, uint32_t b, uint32_t &lo, uint32_t &hi) {
    const unsigned long long p = (unsigned long long)a * b;
    lo = (uint32_t)p;
    hi = (uint32_t)(p >> 32);
}

// Full 128 x 128 -> 256-bit schoolbook product (Eq. 5 on 32-bit words).  The 16 limb products
// are accumulated in two carry chains: E takes the products of the even limbs a0, a2 and O those
// of the odd limbs a1, a3, so that within one row (one limb b_i) the lo and hi halves of a chain
// land in consecutive columns.  Row 0 needs no additions; every later row ends in a fresh limb
// (hi half plus the incoming carry, which cannot overflow), so no separate carry propagation is
// needed.  A final 7-limb addition merges the two chains: 32 multiply instructions and 7 adds.
__device__ __forceinline__ void mul_wide(const uint4 a, const uint4 b, uint32_t c[8]) {
    uint32_t E0, E1, E2, E3, E4, E5, E6, O1, O2, O3, O4, O5, O6, O7;
    mul_wide32(a.x, b.x, E0, E1);  // row 0: four disjoint 64-bit products, no additions
    mul_wide32(a.z, b.x, E2, E3);
    mul_wide32(a.y, b.x, O1, O2);
    mul_wide32(a.w, b.x, O3, O4);
#define MQ_ROW(e0, e1, e2, e3, o1, o2, o3, o4, bi)                                            \
    asm("mad.lo.cc.u32  %0, %8, %12, %0;\n\t"                                                 \
        "madc.hi.cc.u32 %1, %8, %12, %1;\n\t"                                                 \
        "madc.lo.cc.u32 %2, %10, %12, %2;\n\t"                                                \
        "madc.hi.u32    %3, %10, %12, 0;\n\t"                                                 \
        "mad.lo.cc.u32  %4, %9, %12, %4;\n\t"                                                 \
        "madc.hi.cc.u32 %5, %9, %12, %5;\n\t"                                                 \
        "madc.lo.cc.u32 %6, %11, %12, %6;\n\t"                                                \
        "madc.hi.u32    %7, %11, %12, 0;"                                                       \
        : "+r"(e0), "+r"(e1), "+r"(e2), "=r"(e3), "+r"(o1), "+r"(o2), "+r"(o3), "=r"(o4)       \
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(bi));
    MQ_ROW(E1, E2, E3, E4, O2, O3, O4, O5, b.y)
    MQ_ROW(E2, E3, E4, E5, O3, O4, O5, O6, b.z)
    MQ_ROW(E3, E4, E5, E6, O4, O5, O6, O7, b.w)
#undef MQ_ROW
    c[0] = E0;
    asm("add.cc.u32  %0, %7, %13;\n\t"
        "addc.cc.u32 %1, %8, %14;\n\t"
        "addc.cc.u32 %2, %9, %15;\n\t"
        "addc.cc.u32 %3, %10, %16;\n\t"
        "addc.cc.u32 %4, %11, %17;\n\t"
        "addc.cc.u32 %5, %12, %18;\n\t"
        "addc.u32    %6, %19, 0;"
        : "=r"(c[1]), "=r"(c[2]), "=r"(c[3]), "=r"(c[4]), "=r"(c[5]), "=r"(c[6]), "=r"(c[7])
        : "r"(E1), "r"(E2), "r"(E3), "r"(E4), "r"(E5), "r"(E6), "r"(O1), "r"(O2), "r"(O3), "r"(O4), "r"(O5),
          "r"(O6), "r"(O7));
}

// Low 128 bits of a * b: only the products that reach columns 0..3.
__device__ __forceinline__ uint4 mul_lo(const uint4 a, const uint4 b) {
    uint32_t e0, e1, e2, e3, o1, o2, o3;
    // row 0: a0 b0 -> 0, 1; a2 b0 -> 2, 3; a1 b0 -> 1, 2; lo(a3 b0) -> 3
    mul_wide32(a.x, b.x, e0, e1);
    mul_wide32(a.z, b.x, e2, e3);
    mul_wide32(a.y, b.x, o1, o2);
    o3 = a.w * b.x;
    asm("mad.lo.cc.u32  %0, %3, %5, %0;\n\t"
        "madc.hi.cc.u32 %1, %3, %5, %1;\n\t"
        "madc.lo.u32    %2, %4, %5, %2;"
        : "+r"(e1), "+r"(e2), "+r"(e3)
        : "r"(a.x), "r"(a.z), "r"(b.y));
    asm("mad.lo.cc.u32  %0, %2, %3, %0;\n\t"
        "madc.hi.u32    %1, %2, %3, %1;"
        : "+r"(e2), "+r"(e3)
        : "r"(a.x), "r"(b.z));
    asm("mad.lo.u32 %0, %1, %2, %0;" : "+r"(e3) : "r"(a.x), "r"(b.w));
    // odd limbs (a1, a3), one column up
    asm("mad.lo.cc.u32  %0, %2, %3, %0;\n\t"
        "madc.hi.u32    %1, %2, %3, %1;"
        : "+r"(o2), "+r"(o3)
        : "r"(a.y), "r"(b.y));
    asm("mad.lo.u32 %0, %1, %2, %0;" : "+r"(o3) : "r"(a.y), "r"(b.z));
    uint4 r;
    asm("add.cc.u32  %0, %3, %6;\n\t"
        "addc.cc.u32 %1, %4, %7;\n\t"
        "addc.u32    %2, %5, %8;"
        : "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "r"(e1), "r"(e2), "r"(e3), "r"(o1), "r"(o2), "r"(o3));
    r.x = e0;
    return r;
}

// a * w mod q with w' = floor(w * 2^128 / q); a < 2^128, w < q < 2^124.
__device__ __forceinline__ uint4 mul_mod_shoup(uint4 a, uint4 w, uint4 wp, uint4 q) {
    uint32_t h[8];
    mul_wide(a, wp, h);
    uint4 qhat = make_uint4(h[4], h[5], h[6], h[7]);
    uint32_t m;
    uint4 r = sub128(mul_lo(a, w), mul_lo(qhat, q), m);  // true remainder or + q; exact mod 2^128
    return reduce_once(r, q);
}

// floor((a * b - D) / 2^128) where D = a0 b0 + 2^32 (a0 b1 + a1 b0) < 2^98: the high half of the
// product without the three limb products that only reach columns 0..2.  Since D < 2^128 the
// result is the true high half or one less.  26 multiply instructions instead of 32 (13 of them
// high halves instead of 16), in the even/odd chains of mul_wide.
__device__ __forceinline__ uint4 mul_hi_trunc(const uint4 a, const uint4 b) {
    uint32_t E2, E3, E4, E5, E6, O2, O3, O4, O5, O6, O7, h11;
    // row 0 (b0): only a2 b0 -> columns 2, 3 and a3 b0 -> columns 3, 4
    mul_wide32(a.z, b.x, E2, E3);
    mul_wide32(a.w, b.x, O3, O4);
    // row 1 (b1): a2 b1 -> 3, 4 (even chain); a1 b1 -> 2, 3 and a3 b1 -> 4, 5 (odd chain)
    mul_wide32(a.y, b.y, O2, h11);
    asm("mad.lo.cc.u32  %0, %5, %7, %0;\n\t"
        "madc.hi.u32    %1, %5, %7, 0;\n\t"
        "add.cc.u32     %2, %2, %6;\n\t"
        "madc.lo.cc.u32 %3, %8, %7, %3;\n\t"
        "madc.hi.u32    %4, %8, %7, 0;"
        : "+r"(E3), "=r"(E4), "+r"(O3), "+r"(O4), "=r"(O5)
        : "r"(a.z), "r"(h11), "r"(b.y), "r"(a.w));
#define MQ_ROW(e0, e1, e2, e3, o1, o2, o3, o4, bi)                                            \
    asm("mad.lo.cc.u32  %0, %8, %12, %0;\n\t"                                                 \
        "madc.hi.cc.u32 %1, %8, %12, %1;\n\t"                                                 \
        "madc.lo.cc.u32 %2, %10, %12, %2;\n\t"                                                \
        "madc.hi.u32    %3, %10, %12, 0;\n\t"                                                 \
        "mad.lo.cc.u32  %4, %9, %12, %4;\n\t"                                                 \
        "madc.hi.cc.u32 %5, %9, %12, %5;\n\t"                                                 \
        "madc.lo.cc.u32 %6, %11, %12, %6;\n\t"                                                \
        "madc.hi.u32    %7, %11, %12, 0;"                                                       \
        : "+r"(e0), "+r"(e1), "+r"(e2), "=r"(e3), "+r"(o1), "+r"(o2), "+r"(o3), "=r"(o4)       \
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(bi));
    MQ_ROW(E2, E3, E4, E5, O3, O4, O5, O6, b.z)
    MQ_ROW(E3, E4, E5, E6, O4, O5, O6, O7, b.w)
#undef MQ_ROW
    uint4 r;
    uint32_t c2, c3;
    asm("add.cc.u32  %0, %6, %12;\n\t"
        "addc.cc.u32 %1, %7, %13;\n\t"
        "addc.cc.u32 %2, %8, %14;\n\t"
        "addc.cc.u32 %3, %9, %15;\n\t"
        "addc.cc.u32 %4, %10, %16;\n\t"
        "addc.u32    %5, %11, %17;"
        : "=r"(c2), "=r"(c3), "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "r"(E2), "r"(E3), "r"(E4), "r"(E5), "r"(E6), "r"(0u), "r"(O2), "r"(O3), "r"(O4), "r"(O5), "r"(O6),
          "r"(O7));
    (void)c2;
    (void)c3;
    return r;
}

// a * w mod q up to two multiples of q: the result is in [0, 3q).  Shoup's quotient estimate is the
// true quotient or one less, and the truncated high half takes at most one more away.  a may be any
// value below 2^128 (lazy butterflies feed it values below 8q).
__device__ __forceinline__ uint4 mul_mod_shoup_lazy(uint4 a, uint4 w, uint4 wp, uint4 q) {
    uint4 qhat = mul_hi_trunc(a, wp);
    uint32_t m;
    return sub128(mul_lo(a, w), mul_lo(qhat, q), m);  // exact: a w - qhat q < 3q < 2^126
}

// a >= m ? a - m : a
__device__ __forceinline__ uint4 csub(uint4 a, uint4 m) { return reduce_once(a, m); }

__device__ __forceinline__ uint4 add_nored(uint4 a, uint4 b) { return add128(a, b); }

// a + b2 - c for values that keep the result in [0, 2^128): b2 = 2q, c < 2q
__device__ __forceinline__ uint4 add_sub(uint4 a, uint4 b2, uint4 c) {
    uint32_t m;
    return sub128(add128(a, b2), c, m);
}

// floor(c / 2^s) for an 8-limb c whose quotient fits in 128 bits; s uniform across the warp.
__device__ __forceinline__ uint4 shr256(const uint32_t c[8], int s) {
    int sh = s & 31;
    uint4 r;
#define MQ_SHR_CASE(o)                                                                  \
    r.x = __funnelshift_r(c[o + 0], c[o + 1], sh);                                      \
    r.y = __funnelshift_r(c[o + 1], c[o + 2], sh);                                      \
    r.z = __funnelshift_r(c[o + 2], c[o + 3], sh);                                      \
    r.w = __funnelshift_r(c[o + 3], (o + 4 < 8) ? c[(o + 4) & 7] : 0u, sh);
    switch (s >> 5) {
    case 0: MQ_SHR_CASE(0) break;
    case 1: MQ_SHR_CASE(1) break;
    case 2: MQ_SHR_CASE(2) break;
    case 3: MQ_SHR_CASE(3) break;
    default: MQ_SHR_CASE(4) break;
    }
#undef MQ_SHR_CASE
    return r;
}

// a * b mod q for any a, b < q (Barrett, Sec. 2.1).
__device__ __forceinline__ uint4 mul_mod_barrett(uint4 a, uint4 b, const Mod128 &m) {
    uint32_t x[8], t[8];
    mul_wide(a, b, x);                 // x < q^2 < 2^(2L)
    uint4 q1 = shr256(x, m.L - 1);     // < 2^(L+1)
    mul_wide(q1, m.mu, t);             // < 2^(2L+2)
    uint4 q3 = shr256(t, m.L + 1);     // true quotient minus 0, 1 or 2
    uint32_t bm;
    uint4 r = sub128(make_uint4(x[0], x[1], x[2], x[3]), mul_lo(q3, m.q), bm);  // < 3q < 2^126
    r = reduce_once(r, m.q);
    return reduce_once(r, m.q);
}

}  // namespace mq

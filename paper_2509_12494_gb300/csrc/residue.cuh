// residue.cuh -- modular arithmetic on 64-bit and 128-bit residues for sm_103a.
//
// 128-bit values are uint4 = four 32-bit limbs, x lowest (the memory image of a little-endian
// unsigned 128-bit integer, i.e. {lo word, hi word}).  Word operations follow the double-word
// arithmetic of Sec. 2.2: additions with carry and subtractions with borrow are PTX carry chains
// (add.cc/addc, sub.cc/subc -- the GPU's native form of the adc/sbb instructions that MQX adds to
// AVX-512, Table 2), and products use the widening multiply halves mul.lo/mul.hi fused into
// mad.lo.cc/madc.hi.cc chains (schoolbook, Eq. 8).
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

// a * w mod q up to one multiple of q: in [0, 2q) (the final Shoup correction skipped).  nq = -q
// mod 2^64 is not needed here: the compiler's 64-bit high product and one multiply-subtract measured
// faster than a truncated high product with the remainder as a w + qhat nq.
__device__ __forceinline__ uint64_t mul_mod_shoup_lazy(uint64_t a, uint64_t w, uint64_t wp, uint64_t q, uint64_t nq) {
    (void)nq;
    return a * w - __umul64hi(a, wp) * q;
}
__device__ __forceinline__ uint64_t neg(uint64_t q) { return 0 - q; }
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

// r = a - b mod 2^128, where the caller needs no borrow.
__device__ __forceinline__ uint4 sub128(uint4 a, uint4 b) {
    uint4 r;
    asm("sub.cc.u32  %0, %4, %8;\n\t"
        "subc.cc.u32 %1, %5, %9;\n\t"
        "subc.cc.u32 %2, %6, %10;\n\t"
        "subc.u32    %3, %7, %11;"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
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

// Full 128 x 128 -> 256-bit schoolbook product (Eq. 8 on 32-bit words).  Each 32 x 32 -> 64 limb
// product a_j b_i is added into a pair of consecutive columns (i + j, i + j + 1) by a mad.lo.cc /
// madc.hi.cc pair, which the GPU executes as one wide multiply-add on an aligned register pair.
// To keep every pair aligned the products are split by the parity of i + j: E holds the pairs
// (0,1), (2,3), (4,5), (6,7) and takes the products with i + j even, O holds (1,2), (3,4), (5,6),
// (7,8) and takes those with i + j odd, so a chain never has to move its columns by one.  Within
// a chain a row of two products either ends in a column not written before (its high half plus
// the incoming carry cannot overflow) or hands its carry to the next, still empty, column.  A final
// 7-limb addition merges E and O: 32 multiply instructions and 9 adds.
__device__ __forceinline__ void mul_wide(const uint4 a, const uint4 b, uint32_t c[8]) {
    uint32_t E0, E1, E2, E3, E4, E5, E6, E7, O1, O2, O3, O4, O5, O6, O7;
    // b0: a0 b0 -> E(0,1), a2 b0 -> E(2,3), a1 b0 -> O(1,2), a3 b0 -> O(3,4); no additions
    mul_wide32(a.x, b.x, E0, E1);
    mul_wide32(a.z, b.x, E2, E3);
    mul_wide32(a.y, b.x, O1, O2);
    mul_wide32(a.w, b.x, O3, O4);
    // b1: a1 b1 -> E(2,3), a3 b1 -> E(4,5) (new); a0 b1 -> O(1,2), a2 b1 -> O(3,4), carry -> O5
    asm("mad.lo.cc.u32  %0, %4, %6, %0;\n\t"
        "madc.hi.cc.u32 %1, %4, %6, %1;\n\t"
        "madc.lo.cc.u32 %2, %5, %6, 0;\n\t"
        "madc.hi.u32    %3, %5, %6, 0;"
        : "+r"(E2), "+r"(E3), "=r"(E4), "=r"(E5)
        : "r"(a.y), "r"(a.w), "r"(b.y));
    asm("mad.lo.cc.u32  %0, %5, %7, %0;\n\t"
        "madc.hi.cc.u32 %1, %5, %7, %1;\n\t"
        "madc.lo.cc.u32 %2, %6, %7, %2;\n\t"
        "madc.hi.cc.u32 %3, %6, %7, %3;\n\t"
        "addc.u32       %4, 0, 0;"
        : "+r"(O1), "+r"(O2), "+r"(O3), "+r"(O4), "=r"(O5)
        : "r"(a.x), "r"(a.z), "r"(b.y));
    // b2: a0 b2 -> E(2,3), a2 b2 -> E(4,5), carry -> E6; a1 b2 -> O(3,4), a3 b2 -> O(5,6) (O6 new)
    asm("mad.lo.cc.u32  %0, %5, %7, %0;\n\t"
        "madc.hi.cc.u32 %1, %5, %7, %1;\n\t"
        "madc.lo.cc.u32 %2, %6, %7, %2;\n\t"
        "madc.hi.cc.u32 %3, %6, %7, %3;\n\t"
        "addc.u32       %4, 0, 0;"
        : "+r"(E2), "+r"(E3), "+r"(E4), "+r"(E5), "=r"(E6)
        : "r"(a.x), "r"(a.z), "r"(b.z));
    asm("mad.lo.cc.u32  %0, %4, %6, %0;\n\t"
        "madc.hi.cc.u32 %1, %4, %6, %1;\n\t"
        "madc.lo.cc.u32 %2, %5, %6, %2;\n\t"
        "madc.hi.u32    %3, %5, %6, 0;"
        : "+r"(O3), "+r"(O4), "+r"(O5), "=r"(O6)
        : "r"(a.y), "r"(a.w), "r"(b.z));
    // b3: a1 b3 -> E(4,5), a3 b3 -> E(6,7) (E7 new); a0 b3 -> O(3,4), a2 b3 -> O(5,6), carry -> O7
    asm("mad.lo.cc.u32  %0, %4, %6, %0;\n\t"
        "madc.hi.cc.u32 %1, %4, %6, %1;\n\t"
        "madc.lo.cc.u32 %2, %5, %6, %2;\n\t"
        "madc.hi.u32    %3, %5, %6, 0;"
        : "+r"(E4), "+r"(E5), "+r"(E6), "=r"(E7)
        : "r"(a.y), "r"(a.w), "r"(b.w));
    asm("mad.lo.cc.u32  %0, %5, %7, %0;\n\t"
        "madc.hi.cc.u32 %1, %5, %7, %1;\n\t"
        "madc.lo.cc.u32 %2, %6, %7, %2;\n\t"
        "madc.hi.cc.u32 %3, %6, %7, %3;\n\t"
        "addc.u32       %4, 0, 0;"
        : "+r"(O3), "+r"(O4), "+r"(O5), "+r"(O6), "=r"(O7)
        : "r"(a.x), "r"(a.z), "r"(b.w));
    c[0] = E0;
    asm("add.cc.u32  %0, %7, %14;\n\t"
        "addc.cc.u32 %1, %8, %15;\n\t"
        "addc.cc.u32 %2, %9, %16;\n\t"
        "addc.cc.u32 %3, %10, %17;\n\t"
        "addc.cc.u32 %4, %11, %18;\n\t"
        "addc.cc.u32 %5, %12, %19;\n\t"
        "addc.u32    %6, %13, %20;"
        : "=r"(c[1]), "=r"(c[2]), "=r"(c[3]), "=r"(c[4]), "=r"(c[5]), "=r"(c[6]), "=r"(c[7])
        : "r"(E1), "r"(E2), "r"(E3), "r"(E4), "r"(E5), "r"(E6), "r"(E7), "r"(O1), "r"(O2), "r"(O3), "r"(O4),
          "r"(O5), "r"(O6), "r"(O7));
}

// Low 128 bits of a * b: only the products that reach columns 0..3, in the parity-split chains
// of mul_wide (E: pairs (0,1), (2,3); O: the pair (1,2) and column 3, which takes only low halves).
__device__ __forceinline__ uint4 mul_lo(const uint4 a, const uint4 b) {
    uint32_t E0, E1, E2, E3, O1, O2, O3;
    mul_wide32(a.x, b.x, E0, E1);  // a0 b0
    mul_wide32(a.z, b.x, E2, E3);  // a2 b0
    mul_wide32(a.y, b.x, O1, O2);  // a1 b0
    O3 = a.w * b.x;                // lo(a3 b0)
    // even: a1 b1 and a0 b2 -> E(2,3) (carries past column 3 are dropped)
    asm("mad.lo.cc.u32  %0, %2, %4, %0;\n\t"
        "madc.hi.u32    %1, %2, %4, %1;\n\t"
        "mad.lo.cc.u32  %0, %3, %5, %0;\n\t"
        "madc.hi.u32    %1, %3, %5, %1;"
        : "+r"(E2), "+r"(E3)
        : "r"(a.y), "r"(a.x), "r"(b.y), "r"(b.z));
    // odd: a0 b1 -> O(1,2) with its carry into column 3; lo(a2 b1), lo(a1 b2), lo(a0 b3) -> O3
    asm("mad.lo.cc.u32  %0, %3, %6, %0;\n\t"
        "madc.hi.cc.u32 %1, %3, %6, %1;\n\t"
        "madc.lo.u32    %2, %4, %6, %2;\n\t"
        "mad.lo.u32     %2, %5, %7, %2;\n\t"
        "mad.lo.u32     %2, %3, %8, %2;"
        : "+r"(O1), "+r"(O2), "+r"(O3)
        : "r"(a.x), "r"(a.z), "r"(a.y), "r"(b.y), "r"(b.z), "r"(b.w));
    uint4 r;
    r.x = E0;
    asm("add.cc.u32  %0, %3, %6;\n\t"
        "addc.cc.u32 %1, %4, %7;\n\t"
        "addc.u32    %2, %5, %8;"
        : "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "r"(E1), "r"(E2), "r"(E3), "r"(O1), "r"(O2), "r"(O3));
    return r;
}

// Low 128 bits of a * b + c * d, all twenty limb products in one pair of parity-split chains (the
// Shoup remainder a w - qhat q is a w + qhat (2^128 - q) mod 2^128, so one chain and one merge
// replace two low products and a subtraction).
__device__ __forceinline__ uint4 mul_lo2(const uint4 a, const uint4 b, const uint4 c, const uint4 d) {
    uint32_t E0, E1, E2, E3, O1, O2, O3;
    mul_wide32(c.x, d.x, E0, E1);  // c0 d0
    mul_wide32(c.z, d.x, E2, E3);  // c2 d0
    mul_wide32(c.y, d.x, O1, O2);  // c1 d0
    O3 = c.w * d.x;                // lo(c3 d0)
    // even: a0 b0 -> E(0,1) and a2 b0 -> E(2,3) in one chain; a1 b1, a0 b2, c1 d1, c0 d2 -> E(2,3)
    asm("mad.lo.cc.u32  %0, %4, %6, %0;\n\t"
        "madc.hi.cc.u32 %1, %4, %6, %1;\n\t"
        "madc.lo.cc.u32 %2, %5, %6, %2;\n\t"
        "madc.hi.u32    %3, %5, %6, %3;"
        : "+r"(E0), "+r"(E1), "+r"(E2), "+r"(E3)
        : "r"(a.x), "r"(a.z), "r"(b.x));
    asm("mad.lo.cc.u32  %0, %2, %6, %0;\n\t"
        "madc.hi.u32    %1, %2, %6, %1;\n\t"
        "mad.lo.cc.u32  %0, %3, %7, %0;\n\t"
        "madc.hi.u32    %1, %3, %7, %1;\n\t"
        "mad.lo.cc.u32  %0, %4, %8, %0;\n\t"
        "madc.hi.u32    %1, %4, %8, %1;\n\t"
        "mad.lo.cc.u32  %0, %5, %9, %0;\n\t"
        "madc.hi.u32    %1, %5, %9, %1;"
        : "+r"(E2), "+r"(E3)
        : "r"(a.y), "r"(a.x), "r"(c.y), "r"(c.x), "r"(b.y), "r"(b.z), "r"(d.y), "r"(d.z));
    // odd: a1 b0, a0 b1, c0 d1 -> O(1,2), each carrying into column 3 with a low half there;
    // the other low halves of column 3: a1 b2, a0 b3, c1 d2, c0 d3
    asm("mad.lo.cc.u32  %0, %3, %10, %0;\n\t"
        "madc.hi.cc.u32 %1, %3, %10, %1;\n\t"
        "madc.lo.u32    %2, %4, %10, %2;\n\t"
        "mad.lo.cc.u32  %0, %5, %11, %0;\n\t"
        "madc.hi.cc.u32 %1, %5, %11, %1;\n\t"
        "madc.lo.u32    %2, %6, %11, %2;\n\t"
        "mad.lo.cc.u32  %0, %7, %14, %0;\n\t"
        "madc.hi.cc.u32 %1, %7, %14, %1;\n\t"
        "madc.lo.u32    %2, %8, %14, %2;\n\t"
        "mad.lo.u32     %2, %3, %12, %2;\n\t"
        "mad.lo.u32     %2, %5, %13, %2;\n\t"
        "mad.lo.u32     %2, %9, %15, %2;\n\t"
        "mad.lo.u32     %2, %7, %16, %2;"
        : "+r"(O1), "+r"(O2), "+r"(O3)
        : "r"(a.y), "r"(a.w), "r"(a.x), "r"(a.z), "r"(c.x), "r"(c.z), "r"(c.y), "r"(b.x), "r"(b.y), "r"(b.z),
          "r"(b.w), "r"(d.y), "r"(d.z), "r"(d.w));
    uint4 r;
    r.x = E0;
    asm("add.cc.u32  %0, %3, %6;\n\t"
        "addc.cc.u32 %1, %4, %7;\n\t"
        "addc.u32    %2, %5, %8;"
        : "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "r"(E1), "r"(E2), "r"(E3), "r"(O1), "r"(O2), "r"(O3));
    return r;
}

__device__ __forceinline__ uint4 neg(uint4 q) { return sub128(make_uint4(0u, 0u, 0u, 0u), q); }

// a * w mod q with w' = floor(w * 2^128 / q); a < 2^128, w < q < 2^124.
__device__ __forceinline__ uint4 mul_mod_shoup(uint4 a, uint4 w, uint4 wp, uint4 q) {
    uint32_t h[8];
    mul_wide(a, wp, h);
    uint4 qhat = make_uint4(h[4], h[5], h[6], h[7]);
    uint4 r = mul_lo2(a, w, qhat, neg(q));  // a w - qhat q: true remainder or + q
    return reduce_once(r, q);
}

// floor((a * b - D) / 2^128) where D = sum of the limb products a_j b_i with i + j <= 2 (they reach
// columns 0..3 only), D < 3 * 2^128 + 2^98: the true high half minus at most 4.  10 limb products
// instead of 16, in the parity-split chains of mul_wide: O takes columns 3..7 from the products
// with i + j = 3 and 5, E columns 4..7 from those with i + j = 4 and 6; column 3 holds only O3,
// which carries nothing upward by itself.
__device__ __forceinline__ uint4 mul_hi_trunc(const uint4 a, const uint4 b) {
    uint32_t E4, E5, E6, E7, O3, O4, O5, O6, O7;
    mul_wide32(a.w, b.x, O3, O4);  // a3 b0
    mul_wide32(a.w, b.y, E4, E5);  // a3 b1
    // b1: a2 b1 -> O(3,4), carry -> O5
    asm("mad.lo.cc.u32  %0, %3, %4, %0;\n\t"
        "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
        "addc.u32       %2, 0, 0;"
        : "+r"(O3), "+r"(O4), "=r"(O5)
        : "r"(a.z), "r"(b.y));
    // b2: a2 b2 -> E(4,5), carry -> E6; a1 b2 -> O(3,4), a3 b2 -> O(5,6) (O6 new)
    asm("mad.lo.cc.u32  %0, %3, %4, %0;\n\t"
        "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
        "addc.u32       %2, 0, 0;"
        : "+r"(E4), "+r"(E5), "=r"(E6)
        : "r"(a.z), "r"(b.z));
    asm("mad.lo.cc.u32  %0, %4, %6, %0;\n\t"
        "madc.hi.cc.u32 %1, %4, %6, %1;\n\t"
        "madc.lo.cc.u32 %2, %5, %6, %2;\n\t"
        "madc.hi.u32    %3, %5, %6, 0;"
        : "+r"(O3), "+r"(O4), "+r"(O5), "=r"(O6)
        : "r"(a.y), "r"(a.w), "r"(b.z));
    // b3: a1 b3 -> E(4,5), a3 b3 -> E(6,7) (E7 new); a0 b3 -> O(3,4), a2 b3 -> O(5,6), carry -> O7
    asm("mad.lo.cc.u32  %0, %4, %6, %0;\n\t"
        "madc.hi.cc.u32 %1, %4, %6, %1;\n\t"
        "madc.lo.cc.u32 %2, %5, %6, %2;\n\t"
        "madc.hi.u32    %3, %5, %6, 0;"
        : "+r"(E4), "+r"(E5), "+r"(E6), "=r"(E7)
        : "r"(a.y), "r"(a.w), "r"(b.w));
    asm("mad.lo.cc.u32  %0, %5, %7, %0;\n\t"
        "madc.hi.cc.u32 %1, %5, %7, %1;\n\t"
        "madc.lo.cc.u32 %2, %6, %7, %2;\n\t"
        "madc.hi.cc.u32 %3, %6, %7, %3;\n\t"
        "addc.u32       %4, 0, 0;"
        : "+r"(O3), "+r"(O4), "+r"(O5), "+r"(O6), "=r"(O7)
        : "r"(a.x), "r"(a.z), "r"(b.w));
    (void)O3;
    uint4 r;
    asm("add.cc.u32  %0, %4, %8;\n\t"
        "addc.cc.u32 %1, %5, %9;\n\t"
        "addc.cc.u32 %2, %6, %10;\n\t"
        "addc.u32    %3, %7, %11;"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "r"(E4), "r"(E5), "r"(E6), "r"(E7), "r"(O4), "r"(O5), "r"(O6), "r"(O7));
    return r;
}

// a * w mod q up to five multiples of q: the result is in [0, 6q).  Shoup's quotient estimate is
// the true quotient or one less, and the truncated high half takes at most four more away.  a may
// be any value below 2^128 (lazy butterflies feed it values below 16q).  nq = 2^128 - q.
__device__ __forceinline__ uint4 mul_mod_shoup_lazy(uint4 a, uint4 w, uint4 wp, uint4 q, uint4 nq) {
    (void)q;
    uint4 qhat = mul_hi_trunc(a, wp);
    return mul_lo2(a, w, qhat, nq);  // a w - qhat q mod 2^128, exact since it is < 6q < 2^127
}

// a >= m ? a - m : a
__device__ __forceinline__ uint4 csub(uint4 a, uint4 m) { return reduce_once(a, m); }

__device__ __forceinline__ uint4 add_nored(uint4 a, uint4 b) { return add128(a, b); }

// a + b2 - c for values that keep the result in [0, 2^128): c <= a + b2
__device__ __forceinline__ uint4 add_sub(uint4 a, uint4 b2, uint4 c) {
    return sub128(add128(a, b2), c);
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
    uint4 r = sub128(make_uint4(x[0], x[1], x[2], x[3]), mul_lo(q3, m.q));  // < 3q < 2^126
    r = reduce_once(r, m.q);
    return reduce_once(r, m.q);
}

}  // namespace mq

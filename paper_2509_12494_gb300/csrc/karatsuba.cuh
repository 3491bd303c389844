// karatsuba.cuh -- the Karatsuba form of the double-word product (Sec. 2.2, Eq. 9) for 128-bit
// residues, an alternative to the schoolbook product of residue.cuh (Eq. 8) that the multiply
// probes compare: three 64 x 64 -> 128 products of the 64-bit halves instead of four, at the price
// of 65-bit middle sums and the additions and subtractions that fold them back.
#pragma once
#include "residue.cuh"

namespace mq {

// (a1 2^32 + a0)(b1 2^32 + b0) as four 32-bit limbs, in the parity-split chains of mul_wide.
__device__ __forceinline__ void mul64x64(uint32_t a0, uint32_t a1, uint32_t b0, uint32_t b1, uint32_t r[4]) {
    uint32_t E0, E1, E2, E3, O1, O2, O3;
    mul_wide32(a0, b0, E0, E1);
    mul_wide32(a1, b1, E2, E3);
    mul_wide32(a1, b0, O1, O2);
    asm("mad.lo.cc.u32  %0, %3, %4, %0;\n\t"
        "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
        "addc.u32       %2, 0, 0;"
        : "+r"(O1), "+r"(O2), "=r"(O3)
        : "r"(a0), "r"(b1));
    r[0] = E0;
    asm("add.cc.u32  %0, %3, %6;\n\t"
        "addc.cc.u32 %1, %4, %7;\n\t"
        "addc.u32    %2, %5, %8;"
        : "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
        : "r"(E1), "r"(E2), "r"(E3), "r"(O1), "r"(O2), "r"(O3));
}

// Full 128 x 128 -> 256-bit product by Eq. 9 on 64-bit halves A = A1 2^64 + A0, B = B1 2^64 + B0:
// P0 = A0 B0, P2 = A1 B1, P1 = (A0 + A1)(B0 + B1) with 65-bit sums (carries ca, cb), and
// A B = P2 2^128 + (P1 - P0 - P2) 2^64 + P0.  P1 < 2^130 takes five limbs; P1 - P0 - P2 =
// A0 B1 + A1 B0 < 2^129 as well.
__device__ __forceinline__ void mul_wide_karatsuba(const uint4 a, const uint4 b, uint32_t c[8]) {
    uint32_t p0[4], p1[4], p2[4];
    mul64x64(a.x, a.y, b.x, b.y, p0);
    mul64x64(a.z, a.w, b.z, b.w, p2);
    uint32_t sa0, sa1, ca, sb0, sb1, cb;
    asm("add.cc.u32  %0, %3, %5;\n\t"
        "addc.cc.u32 %1, %4, %6;\n\t"
        "addc.u32    %2, 0, 0;"
        : "=r"(sa0), "=r"(sa1), "=r"(ca)
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w));
    asm("add.cc.u32  %0, %3, %5;\n\t"
        "addc.cc.u32 %1, %4, %6;\n\t"
        "addc.u32    %2, 0, 0;"
        : "=r"(sb0), "=r"(sb1), "=r"(cb)
        : "r"(b.x), "r"(b.y), "r"(b.z), "r"(b.w));
    mul64x64(sa0, sa1, sb0, sb1, p1);
    // + 2^64 (ca (sb0, sb1) + cb (sa0, sa1)) + 2^128 ca cb
    const uint32_t ma = 0u - ca, mb = 0u - cb;
    uint32_t p14;
    asm("add.cc.u32  %0, %0, %3;\n\t"
        "addc.cc.u32 %1, %1, %4;\n\t"
        "addc.u32    %2, %5, 0;"
        : "+r"(p1[2]), "+r"(p1[3]), "=r"(p14)
        : "r"(sb0 & ma), "r"(sb1 & ma), "r"(ca & cb));
    asm("add.cc.u32  %0, %0, %3;\n\t"
        "addc.cc.u32 %1, %1, %4;\n\t"
        "addc.u32    %2, %2, 0;"
        : "+r"(p1[2]), "+r"(p1[3]), "+r"(p14)
        : "r"(sa0 & mb), "r"(sa1 & mb));
    // middle = P1 - P0 - P2
    uint32_t m0, m1, m2, m3, m4;
    asm("sub.cc.u32  %0, %5, %10;\n\t"
        "subc.cc.u32 %1, %6, %11;\n\t"
        "subc.cc.u32 %2, %7, %12;\n\t"
        "subc.cc.u32 %3, %8, %13;\n\t"
        "subc.u32    %4, %9, 0;"
        : "=r"(m0), "=r"(m1), "=r"(m2), "=r"(m3), "=r"(m4)
        : "r"(p1[0]), "r"(p1[1]), "r"(p1[2]), "r"(p1[3]), "r"(p14), "r"(p0[0]), "r"(p0[1]), "r"(p0[2]), "r"(p0[3]));
    asm("sub.cc.u32  %0, %0, %5;\n\t"
        "subc.cc.u32 %1, %1, %6;\n\t"
        "subc.cc.u32 %2, %2, %7;\n\t"
        "subc.cc.u32 %3, %3, %8;\n\t"
        "subc.u32    %4, %4, 0;"
        : "+r"(m0), "+r"(m1), "+r"(m2), "+r"(m3), "+r"(m4)
        : "r"(p2[0]), "r"(p2[1]), "r"(p2[2]), "r"(p2[3]));
    c[0] = p0[0];
    c[1] = p0[1];
    asm("add.cc.u32  %0, %6, %8;\n\t"
        "addc.cc.u32 %1, %7, %9;\n\t"
        "addc.cc.u32 %2, %10, %12;\n\t"
        "addc.cc.u32 %3, %11, %13;\n\t"
        "addc.cc.u32 %4, %14, %16;\n\t"
        "addc.u32    %5, %15, 0;"
        : "=r"(c[2]), "=r"(c[3]), "=r"(c[4]), "=r"(c[5]), "=r"(c[6]), "=r"(c[7])
        : "r"(p0[2]), "r"(p0[3]), "r"(m0), "r"(m1), "r"(p2[0]), "r"(p2[1]), "r"(m2), "r"(m3), "r"(p2[2]),
          "r"(p2[3]), "r"(m4));
}

// a * b mod q for any a, b < q (Barrett, Sec. 2.1, Eq. 4) with both full products by Eq. 9.
__device__ __forceinline__ uint4 mul_mod_barrett_karatsuba(uint4 a, uint4 b, const Mod128 &m) {
    uint32_t x[8], t[8];
    mul_wide_karatsuba(a, b, x);
    uint4 q1 = shr256(x, m.L - 1);
    mul_wide_karatsuba(q1, m.mu, t);
    uint4 q3 = shr256(t, m.L + 1);
    uint4 r = sub128(make_uint4(x[0], x[1], x[2], x[3]), mul_lo(q3, m.q));
    r = reduce_once(r, m.q);
    return reduce_once(r, m.q);
}

}  // namespace mq

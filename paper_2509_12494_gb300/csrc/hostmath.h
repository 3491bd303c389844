// hostmath.h -- host-side 128-bit scalar arithmetic for plan and call set-up.
//
// Only a handful of values per call go through here (Barrett's mu, Shoup companions of scalars,
// the inverse root, N^-1), so plain binary long division is fast enough.  unsigned __int128 is a
// GCC extension available on x86-64 and aarch64 alike.
#pragma once
#include <stdint.h>

namespace hm {

typedef unsigned __int128 u128;

inline u128 from_words(const uint64_t w[2]) { return ((u128)w[1] << 64) | w[0]; }
inline void to_words(u128 v, uint64_t w[2]) {
    w[0] = (uint64_t)v;
    w[1] = (uint64_t)(v >> 64);
}

inline int bitlen(u128 v) {
    int n = 0;
    while (v) {
        ++n;
        v >>= 1;
    }
    return n;
}

// a * b mod q for a, b < q < 2^126: 256-bit schoolbook product, then the remainder bit by bit.
inline u128 mulmod(u128 a, u128 b, u128 q) {
    uint64_t a0 = (uint64_t)a, a1 = (uint64_t)(a >> 64), b0 = (uint64_t)b, b1 = (uint64_t)(b >> 64);
    u128 p00 = (u128)a0 * b0, p01 = (u128)a0 * b1, p10 = (u128)a1 * b0, p11 = (u128)a1 * b1;
    u128 mid = (p00 >> 64) + (uint64_t)p01 + (uint64_t)p10;  // < 3 * 2^64
    uint64_t w[4];
    w[0] = (uint64_t)p00;
    w[1] = (uint64_t)mid;
    u128 hi = p11 + (p01 >> 64) + (p10 >> 64) + (mid >> 64);
    w[2] = (uint64_t)hi;
    w[3] = (uint64_t)(hi >> 64);
    u128 r = 0;
    for (int i = 255; i >= 0; --i) {
        r = (r << 1) | ((w[i / 64] >> (i % 64)) & 1);
        if (r >= q) r -= q;
    }
    return r;
}

inline u128 powmod(u128 g, u128 e, u128 q) {
    u128 acc = 1 % q, base = g % q;
    for (int i = 127; i >= 0; --i) {
        acc = mulmod(acc, acc, q);
        if ((e >> i) & 1) acc = mulmod(acc, base, q);
    }
    return acc;
}

// floor(2^(2L) / q) with L = bitlen(q) <= 124: the quotient is below 2^(L+1).
inline u128 barrett_mu(u128 q, int L) {
    u128 r = 0, quo = 0;
    for (int i = 2 * L; i >= 0; --i) {
        r = (r << 1) | (i == 2 * L ? 1u : 0u);
        quo <<= 1;
        if (r >= q) {
            r -= q;
            quo |= 1;
        }
    }
    return quo;
}

// floor(w * 2^B / q) for w < q < 2^126 and B = 64 or 128 (Shoup's companion of a fixed multiplier).
inline u128 shoup(u128 w, u128 q, int B) {
    u128 r = w, quo = 0;
    for (int i = 0; i < B; ++i) {
        r <<= 1;
        quo <<= 1;
        if (r >= q) {
            r -= q;
            quo |= 1;
        }
    }
    return quo;
}

}  // namespace hm

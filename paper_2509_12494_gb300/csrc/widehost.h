// widehost.h -- host arithmetic on integers of up to 512 bits (8 little-endian 64-bit words) for the
// constants of plans and BLAS calls on residues of three and four words: modular products and
// powers by schoolbook products and binary long division, Barrett's mu and Shoup companions by
// bit-serial division.  Slow and simple; it runs once per plan.
#pragma once
#include <stdint.h>
#include <string.h>

namespace hw {

typedef unsigned __int128 u128;

struct U {
    uint64_t w[8];
};

inline U zero() {
    U r;
    memset(&r, 0, sizeof r);
    return r;
}

inline U from_words(const uint64_t *v, int n) {
    U r = zero();
    for (int k = 0; k < n; ++k) r.w[k] = v[k];
    return r;
}

inline U from_u64(uint64_t v) { return from_words(&v, 1); }

inline void to_words(const U &a, uint64_t *v, int n) {
    for (int k = 0; k < n; ++k) v[k] = a.w[k];
}

inline int cmp(const U &a, const U &b) {
    for (int k = 7; k >= 0; --k)
        if (a.w[k] != b.w[k]) return a.w[k] < b.w[k] ? -1 : 1;
    return 0;
}

inline U add(const U &a, const U &b) {
    U r;
    uint64_t c = 0;
    for (int k = 0; k < 8; ++k) {
        u128 t = (u128)a.w[k] + b.w[k] + c;
        r.w[k] = (uint64_t)t;
        c = (uint64_t)(t >> 64);
    }
    return r;
}

inline U sub(const U &a, const U &b) {  // a >= b
    U r;
    uint64_t br = 0;
    for (int k = 0; k < 8; ++k) {
        u128 t = (u128)a.w[k] - b.w[k] - br;
        r.w[k] = (uint64_t)t;
        br = (uint64_t)(t >> 64) & 1u;
    }
    return r;
}

inline int bitlen(const U &a) {
    for (int k = 7; k >= 0; --k)
        if (a.w[k]) return 64 * k + 64 - __builtin_clzll(a.w[k]);
    return 0;
}

inline int bit(const U &a, int i) { return (int)((a.w[i / 64] >> (i % 64)) & 1u); }

inline U shl1(const U &a) {
    U r;
    for (int k = 7; k > 0; --k) r.w[k] = (a.w[k] << 1) | (a.w[k - 1] >> 63);
    r.w[0] = a.w[0] << 1;
    return r;
}

inline U shr(const U &a, int s) {  // s < 64
    if (s == 0) return a;
    U r;
    for (int k = 0; k < 7; ++k) r.w[k] = (a.w[k] >> s) | (a.w[k + 1] << (64 - s));
    r.w[7] = a.w[7] >> s;
    return r;
}

// a * b for a, b < 2^256
inline U mul(const U &a, const U &b) {
    U r = zero();
    for (int i = 0; i < 4; ++i) {
        uint64_t c = 0;
        for (int j = 0; j < 4; ++j) {
            u128 t = (u128)a.w[j] * b.w[i] + r.w[i + j] + c;
            r.w[i + j] = (uint64_t)t;
            c = (uint64_t)(t >> 64);
        }
        r.w[i + 4] = c;
    }
    return r;
}

// x mod q by binary long division, q > 0, q < 2^256
inline U mod(const U &x, const U &q) {
    U r = zero();
    for (int i = bitlen(x) - 1; i >= 0; --i) {
        r = shl1(r);
        r.w[0] |= (uint64_t)bit(x, i);
        if (cmp(r, q) >= 0) r = sub(r, q);
    }
    return r;
}

inline U mulmod(const U &a, const U &b, const U &q) { return mod(mul(a, b), q); }

inline U powmod(const U &g, uint64_t e, const U &q) {
    U acc = mod(from_u64(1), q), base = mod(g, q);
    for (int i = 63; i >= 0; --i) {
        acc = mulmod(acc, acc, q);
        if ((e >> i) & 1) acc = mulmod(acc, base, q);
    }
    return acc;
}

// floor(2^(2L) / q)
inline U barrett_mu(const U &q, int L) {
    U r = zero(), quo = zero();
    for (int i = 2 * L; i >= 0; --i) {
        r = shl1(r);
        if (i == 2 * L) r.w[0] |= 1;
        quo = shl1(quo);
        if (cmp(r, q) >= 0) {
            r = sub(r, q);
            quo.w[0] |= 1;
        }
    }
    return quo;
}

// floor(w * 2^B / q) for w < q (Shoup's companion of a fixed multiplier)
inline U shoup(const U &w, const U &q, int B) {
    U r = w, quo = zero();
    for (int i = 0; i < B; ++i) {
        r = shl1(r);
        quo = shl1(quo);
        if (cmp(r, q) >= 0) {
            r = sub(r, q);
            quo.w[0] |= 1;
        }
    }
    return quo;
}

}  // namespace hw

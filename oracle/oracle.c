/*
 * oracle.c -- plain CPU reference for modular BLAS and the number theoretic transform.
 *
 * TEST INFRASTRUCTURE, NOT PART OF THE LIBRARY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file's shared object.  The CUDA library never
 * includes, links or calls anything here, and nothing here is shared with it.
 *
 * Every operation is computed from its textbook definition with an arbitrary-precision integer of
 * 32-bit limbs: schoolbook products and binary long division (shift-and-subtract, one quotient bit
 * per step).  There is no Barrett, Montgomery or Shoup reduction, no carry trick and no lazy
 * reduction.  The paper's reading of each function is cited beside it:
 *
 *   Sec. 2.1, Eq. 1       ring operations c = a + b, a - b, ab mod q on Z_q
 *   Sec. 2.3              point-wise polynomial ops as BLAS (vector add/sub/multiply, axpy y = ax + y)
 *   Sec. 2.3, Eq. 11      n-point NTT y_k = sum_j x_j w^{jk} mod q (cyclic, natural order)
 *   Sec. 2.3              schoolbook polynomial product
 *   Sec. 3.2 (last par.)  butterfly = one modular add, one modular sub, one modular mul;
 *                         log n stages of n/2 butterflies
 *
 * Residues are passed as arrays of 64-bit words: width w = w words per residue, low word first
 * (width 1: q < 2^64; width 2: the memory order of an unsigned 128-bit value).  Moduli and roots
 * are arrays of max(w, 2) words.  The default build takes widths 1 and 2; the wide build
 * (-DBN_LIMBS=18) also takes widths 3 and 4 (residues of 192 and 256 bits, the larger bit-widths
 * of Sec. 7), with the same code on longer integers.
 *
 * Readings of the paper taken here (each one a choice where the paper is silent):
 *   - the negacyclic transform (modulus x^N + 1) with a primitive 2N-th root psi is
 *     yhat_k = sum_j x_j psi^{(2k+1) j}, i.e. the cyclic transform with w = psi^2 of (x_j psi^j);
 *   - the inverse transform includes the factor N^{-1} (and psi^{-j}), so inverse(forward(x)) = x;
 *   - "bit-reversed order" output stores yhat_{brv(i)} at position i; the inverse in that order
 *     reads its input the same way;
 *   - vsub computes a - b; axpy computes s*x + y.
 * Parity is pinned for every exported function (see the header comment of each).
 */
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#ifndef BN_LIMBS
#define BN_LIMBS 10 /* 320 bits: a product of two values below 2^128 needs 8 limbs */
#endif
/* widths the build takes: a product of two values below 2^(64 w) needs 4 w limbs, plus one */
#define MAX_WIDTH ((BN_LIMBS - 1) / 4)

typedef struct {
    uint32_t l[BN_LIMBS]; /* little-endian 32-bit limbs */
} bn;

/* ---------------------------------------------------------------- multi-precision integers */

/* a = the nw 64-bit words w[0..nw-1], low word first */
static void bn_set_words(bn *a, const uint64_t *w, int nw) {
    memset(a, 0, sizeof *a);
    for (int k = 0; k < nw; ++k) {
        a->l[2 * k] = (uint32_t)w[k];
        a->l[2 * k + 1] = (uint32_t)(w[k] >> 32);
    }
}

static void bn_set_u64(bn *a, uint64_t v) { bn_set_words(a, &v, 1); }

static void bn_get_words(const bn *a, uint64_t *w, int nw) {
    for (int k = 0; k < nw; ++k) w[k] = (uint64_t)a->l[2 * k] | ((uint64_t)a->l[2 * k + 1] << 32);
}

static int bn_cmp(const bn *a, const bn *b) {
    for (int i = BN_LIMBS - 1; i >= 0; --i) {
        if (a->l[i] != b->l[i]) return a->l[i] < b->l[i] ? -1 : 1;
    }
    return 0;
}

/* r = a + b (the caller guarantees no overflow of BN_LIMBS limbs) */
static void bn_add(bn *r, const bn *a, const bn *b) {
    uint64_t carry = 0;
    for (int i = 0; i < BN_LIMBS; ++i) {
        uint64_t s = (uint64_t)a->l[i] + b->l[i] + carry;
        r->l[i] = (uint32_t)s;
        carry = s >> 32;
    }
}

/* r = a - b, requires a >= b */
static void bn_sub(bn *r, const bn *a, const bn *b) {
    uint64_t borrow = 0;
    for (int i = 0; i < BN_LIMBS; ++i) {
        uint64_t d = (uint64_t)a->l[i] - b->l[i] - borrow;
        r->l[i] = (uint32_t)d;
        borrow = (d >> 63) & 1; /* the difference wrapped below zero */
    }
}

/* r = a * b, schoolbook: every limb of a times every limb of b (the caller keeps it in range) */
static void bn_mul(bn *r, const bn *a, const bn *b) {
    uint32_t acc[2 * BN_LIMBS];
    memset(acc, 0, sizeof acc);
    for (int i = 0; i < BN_LIMBS; ++i) {
        uint64_t carry = 0;
        for (int j = 0; j < BN_LIMBS; ++j) {
            uint64_t t = (uint64_t)a->l[i] * b->l[j] + acc[i + j] + carry;
            acc[i + j] = (uint32_t)t;
            carry = t >> 32;
        }
        for (int k = i + BN_LIMBS; carry && k < 2 * BN_LIMBS; ++k) {
            uint64_t t = (uint64_t)acc[k] + carry;
            acc[k] = (uint32_t)t;
            carry = t >> 32;
        }
    }
    memcpy(r->l, acc, sizeof r->l);
}

static int bn_bitlen(const bn *a) {
    for (int i = BN_LIMBS - 1; i >= 0; --i) {
        if (a->l[i]) {
            int b = 32;
            while (!((a->l[i] >> (b - 1)) & 1)) --b;
            return 32 * i + b;
        }
    }
    return 0;
}

static int bn_bit(const bn *a, int i) { return (a->l[i / 32] >> (i % 32)) & 1; }

static void bn_shl1(bn *a) {
    for (int i = BN_LIMBS - 1; i > 0; --i) a->l[i] = (a->l[i] << 1) | (a->l[i - 1] >> 31);
    a->l[0] <<= 1;
}

/* r = x mod q by binary long division: bring down one bit of x at a time, subtract q when the
 * partial remainder reaches it.  q > 0. */
static void bn_mod(bn *r, const bn *x, const bn *q) {
    bn rem;
    memset(&rem, 0, sizeof rem);
    for (int i = bn_bitlen(x) - 1; i >= 0; --i) {
        bn_shl1(&rem);
        rem.l[0] |= (uint32_t)bn_bit(x, i);
        if (bn_cmp(&rem, q) >= 0) bn_sub(&rem, &rem, q);
    }
    *r = rem;
}

/* ---------------------------------------------------------------- Z_q arithmetic (Sec. 2.1, Eq. 1) */

static void mod_add(bn *r, const bn *a, const bn *b, const bn *q) {
    bn s;
    bn_add(&s, a, b);
    bn_mod(r, &s, q);
}

/* (a - b) mod q computed as (a + (q - (b mod q))) mod q, which never goes below zero */
static void mod_sub(bn *r, const bn *a, const bn *b, const bn *q) {
    bn bm, s;
    bn_mod(&bm, b, q);
    bn_sub(&s, q, &bm);
    bn_add(&s, &s, a);
    bn_mod(r, &s, q);
}

static void mod_mul(bn *r, const bn *a, const bn *b, const bn *q) {
    bn p;
    bn_mul(&p, a, b);
    bn_mod(r, &p, q);
}

/* g^e mod q by left-to-right square-and-multiply over the bits of e */
static void mod_pow(bn *r, const bn *g, const bn *e, const bn *q) {
    bn acc, base;
    bn_set_u64(&acc, 1);
    bn_mod(&acc, &acc, q);
    bn_mod(&base, g, q);
    for (int i = bn_bitlen(e) - 1; i >= 0; --i) {
        mod_mul(&acc, &acc, &acc, q);
        if (bn_bit(e, i)) mod_mul(&acc, &acc, &base, q);
    }
    *r = acc;
}

/* inverse of a nonzero a modulo a prime q (Fermat): a^(q-2) */
static void mod_inv(bn *r, const bn *a, const bn *q) {
    bn e, two;
    bn_set_u64(&two, 2);
    bn_sub(&e, q, &two);
    mod_pow(r, a, &e, q);
}

static void mod_pow_u64(bn *r, const bn *g, uint64_t e, const bn *q) {
    bn be;
    bn_set_u64(&be, e);
    mod_pow(r, g, &be, q);
}

/* ---------------------------------------------------------------- element I/O */

static void load_elem(bn *a, const uint64_t *p, size_t i, int width) { bn_set_words(a, p + (size_t)width * i, width); }

static void store_elem(uint64_t *p, size_t i, const bn *a, int width) { bn_get_words(a, p + (size_t)width * i, width); }

/* words of a modulus or root array: max(width, 2) */
static int arg_words(int width) { return width < 2 ? 2 : width; }

static int check_args(const uint64_t *q, int width) {
    if (width < 1 || width > MAX_WIDTH) return -1;
    if (width == 1 && q[1] != 0) return -1;
    int big = 0;
    for (int k = 1; k < arg_words(width); ++k) big |= q[k] != 0;
    if (!big && q[0] < 2) return -1;
    return 0;
}

/* The widest residue (in 64-bit words) this compiled copy takes: 2, or 4 for the wide build. */
int oracle_max_width(void) { return MAX_WIDTH; }

/* ---------------------------------------------------------------- BLAS (Sec. 2.3) */

enum { OR_VADD = 0, OR_VSUB = 1, OR_VMUL = 2, OR_AXPY = 3 };

/*
 * Point-wise vector operations over Z_q, element by element (Sec. 2.3, "Point-wise polynomial
 * operations"; ring operations of Sec. 2.1, Eq. 1):
 *   OR_VADD  out_i = a_i + b_i mod q
 *   OR_VSUB  out_i = a_i - b_i mod q
 *   OR_VMUL  out_i = a_i * b_i mod q
 *   OR_AXPY  out_i = s * a_i + b_i mod q      (axpy y = s x + y with x = a, y = b)
 * `s` is one residue (ignored unless OR_AXPY).  `out` may alias `a` or `b`.
 * Pinned by: Python integers on random and edge operands, and the field identities.
 */
int oracle_blas(int op, uint64_t *out, const uint64_t *a, const uint64_t *b, const uint64_t *s,
                size_t n, const uint64_t *q, int width) {
    if (check_args(q, width) || op < 0 || op > 3) return -1;
    bn Q, A, B, S, R;
    bn_set_words(&Q, q, arg_words(width));
    if (op == OR_AXPY) load_elem(&S, s, 0, width);
    for (size_t i = 0; i < n; ++i) {
        load_elem(&A, a, i, width);
        load_elem(&B, b, i, width);
        switch (op) {
        case OR_VADD: mod_add(&R, &A, &B, &Q); break;
        case OR_VSUB: mod_sub(&R, &A, &B, &Q); break;
        case OR_VMUL: mod_mul(&R, &A, &B, &Q); break;
        default: {
            bn T;
            mod_mul(&T, &S, &A, &Q);
            mod_add(&R, &T, &B, &Q);
        }
        }
        store_elem(out, i, &R, width);
    }
    return 0;
}

/* ---------------------------------------------------------------- NTT (Sec. 2.3, Eq. 11) */

#define OR_CYCLIC 1u /* root is an N-th root w; otherwise a 2N-th root psi (negacyclic) */
#define OR_BITREV 2u /* transformed side in bit-reversed order */

static size_t bit_reverse(size_t i, unsigned bits) {
    size_t r = 0;
    for (unsigned b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}

static void permute_bit_reversed(bn *A, unsigned log2n) {
    size_t N = (size_t)1 << log2n;
    for (size_t i = 0; i < N; ++i) {
        size_t j = bit_reverse(i, log2n);
        if (i < j) {
            bn t = A[i];
            A[i] = A[j];
            A[j] = t;
        }
    }
}

/*
 * Cyclic transform A_k <- sum_j A_j w^{jk} mod q in natural order, by the textbook iterative
 * radix-2 Cooley-Tukey algorithm: a bit-reversal permutation of the input, then log2 N stages;
 * stage s combines pairs at distance m/2 (m = 2^s) with the butterfly
 *   (u, t) = (A[k+j], w_m^j * A[k+j+m/2]);  A[k+j] = u + t;  A[k+j+m/2] = u - t,
 * w_m = w^{N/m}.  Each butterfly is one modular mul, add and sub (Sec. 3.2, last paragraph).
 */
static void cyclic_transform(bn *A, unsigned log2n, const bn *w, const bn *Q, bn *pw) {
    size_t N = (size_t)1 << log2n;
    permute_bit_reversed(A, log2n);
    for (unsigned s = 1; s <= log2n; ++s) {
        size_t m = (size_t)1 << s, half = m / 2;
        bn wm;
        mod_pow_u64(&wm, w, N / m, Q);
        bn_set_u64(&pw[0], 1);
        for (size_t j = 1; j < half; ++j) mod_mul(&pw[j], &pw[j - 1], &wm, Q);
        for (size_t k = 0; k < N; k += m) {
            for (size_t j = 0; j < half; ++j) {
                bn u = A[k + j], t;
                mod_mul(&t, &pw[j], &A[k + j + half], Q);
                mod_add(&A[k + j], &u, &t, Q);
                mod_sub(&A[k + j + half], &u, &t, Q);
            }
        }
    }
}

/*
 * In-place transform of one polynomial of N = 2^log2n residues.
 *   forward, cyclic:       y_k = sum_j x_j w^{jk}                         (Eq. 11)
 *   forward, negacyclic:   y_k = sum_j x_j psi^{(2k+1) j}  = cyclic_{w=psi^2}(x_j psi^j)_k
 *   inverse, cyclic:       x_j = N^{-1} sum_k y_k w^{-jk}
 *   inverse, negacyclic:   x_j = N^{-1} psi^{-j} sum_k y_k psi^{-2jk}
 * With OR_BITREV the transformed side (forward output, inverse input) is in bit-reversed order.
 * `work` must hold 2 * N / 2 + N bn values (caller-provided scratch, see oracle_ntt).
 * q must be prime (the inverse uses Fermat) and root of the stated order.
 * Pinned by: the worked example of Sec. 2.3, brute-force DFT with Python integers for N <= 64,
 * closed forms (unit vectors), inverse(forward(x)) = x, the convolution theorem against the
 * schoolbook product, and Python-integer spot checks of single outputs.
 */
static void ntt_one(uint64_t *x, unsigned log2n, const bn *Q, const bn *root, int width,
                    unsigned flags, int inverse, bn *A, bn *pw) {
    size_t N = (size_t)1 << log2n;
    int cyclic = (flags & OR_CYCLIC) != 0;
    bn w, psi_inv, n_inv, N_bn, f, t;
    for (size_t i = 0; i < N; ++i) load_elem(&A[i], x, i, width);

    if (cyclic)
        w = *root;
    else
        mod_mul(&w, root, root, Q); /* w = psi^2 */

    if (!inverse) {
        if (!cyclic) { /* twist: x_j * psi^j */
            bn_set_u64(&f, 1);
            for (size_t j = 0; j < N; ++j) {
                mod_mul(&A[j], &A[j], &f, Q);
                mod_mul(&f, &f, root, Q);
            }
        }
        cyclic_transform(A, log2n, &w, Q, pw);
        if (flags & OR_BITREV) permute_bit_reversed(A, log2n);
    } else {
        if (flags & OR_BITREV) permute_bit_reversed(A, log2n);
        bn w_inv;
        mod_inv(&w_inv, &w, Q);
        cyclic_transform(A, log2n, &w_inv, Q, pw);
        bn_set_u64(&N_bn, (uint64_t)N);
        mod_inv(&n_inv, &N_bn, Q);
        if (cyclic) {
            for (size_t j = 0; j < N; ++j) mod_mul(&A[j], &A[j], &n_inv, Q);
        } else { /* untwist: N^{-1} psi^{-j} */
            mod_inv(&psi_inv, root, Q);
            f = n_inv;
            for (size_t j = 0; j < N; ++j) {
                mod_mul(&t, &A[j], &f, Q);
                A[j] = t;
                mod_mul(&f, &f, &psi_inv, Q);
            }
        }
    }
    for (size_t i = 0; i < N; ++i) store_elem(x, i, &A[i], width);
}

/*
 * Batched in-place transform: `batch` polynomials, polynomial b starting at residue b * stride.
 * `work` is caller-owned scratch of at least oracle_ntt_work_bytes(log2n) bytes (the oracle does
 * no allocation, so the caller's threads can each pass their own).
 * Returns 0, or -1 on bad arguments.
 */
size_t oracle_ntt_work_bytes(unsigned log2n) { return sizeof(bn) * (((size_t)3 << log2n) / 2 + 1); }

int oracle_ntt(uint64_t *x, size_t batch, size_t stride, unsigned log2n, const uint64_t *q,
               const uint64_t *root, int width, unsigned flags, int inverse, void *work) {
    if (check_args(q, width) || log2n > 24 || !work) return -1;
    size_t N = (size_t)1 << log2n;
    if (batch > 1 && stride < N) return -1;
    bn Q, R;
    bn_set_words(&Q, q, arg_words(width));
    bn_set_words(&R, root, arg_words(width));
    bn *A = (bn *)work, *pw = A + N;
    for (size_t b = 0; b < batch; ++b)
        ntt_one(x + b * stride * (size_t)width, log2n, &Q, &R, width, flags, inverse, A, pw);
    return 0;
}

/*
 * The same transforms straight from the definition, O(N^2), for small N (Eq. 11 and the negacyclic
 * reading above).  out must not alias x.  Flags as in oracle_ntt.
 * Pinned by: the worked example of Sec. 2.3 and the unit-vector closed forms.
 */
int oracle_dft(uint64_t *out, const uint64_t *x, unsigned log2n, const uint64_t *q,
               const uint64_t *root, int width, unsigned flags, int inverse) {
    if (check_args(q, width) || log2n > 12) return -1;
    size_t N = (size_t)1 << log2n;
    int cyclic = (flags & OR_CYCLIC) != 0;
    /* order of the root: N (cyclic) or 2N (negacyclic); exponents are reduced modulo it */
    size_t ord = cyclic ? N : 2 * N;
    bn Q, g, acc, term, xe, e, scale, N_bn;
    bn_set_words(&Q, q, arg_words(width));
    bn_set_words(&g, root, arg_words(width));
    if (inverse) mod_inv(&g, &g, &Q);
    bn_set_u64(&N_bn, (uint64_t)N);
    mod_inv(&scale, &N_bn, &Q);
    for (size_t o = 0; o < N; ++o) {     /* natural index of the output */
        bn_set_u64(&acc, 0);
        for (size_t i = 0; i < N; ++i) { /* natural index of the summed input */
            /* forward: output k = o, sum over coefficients j = i;
               inverse: output j = o, sum over frequencies k = i */
            size_t j = inverse ? o : i, k = inverse ? i : o;
            uint64_t ex = cyclic ? (uint64_t)((j * k) % ord) : (uint64_t)(((2 * k + 1) * j) % ord);
            /* a bit-reversed input holds element i at position brv(i) */
            size_t src = (inverse && (flags & OR_BITREV)) ? bit_reverse(i, log2n) : i;
            mod_pow_u64(&e, &g, ex, &Q);
            load_elem(&xe, x, src, width);
            mod_mul(&term, &xe, &e, &Q);
            mod_add(&acc, &acc, &term, &Q);
        }
        if (inverse) mod_mul(&acc, &acc, &scale, &Q);
        /* a bit-reversed output holds y_k at position brv(k) */
        size_t dst = (!inverse && (flags & OR_BITREV)) ? bit_reverse(o, log2n) : o;
        store_elem(out, dst, &acc, width);
    }
    return 0;
}

/*
 * One output of the forward transform, from the definition, in O(N) modular operations:
 * yhat_k = sum_j x_j r^{e(j)} with r^{e(j)} = (root^{k'})^j, k' = k (cyclic) or 2k+1 (negacyclic).
 * Used to check single outputs of transforms too large for the full oracle.
 * `k` is the natural-order frequency index.
 */
int oracle_ntt_point(uint64_t *out, const uint64_t *x, unsigned log2n, const uint64_t *q,
                     const uint64_t *root, int width, unsigned flags, uint64_t k) {
    if (check_args(q, width) || log2n > 30) return -1;
    size_t N = (size_t)1 << log2n;
    if (k >= N) return -1;
    int cyclic = (flags & OR_CYCLIC) != 0;
    bn Q, g, step, pw, acc, xe, term;
    bn_set_words(&Q, q, arg_words(width));
    bn_set_words(&g, root, arg_words(width));
    mod_pow_u64(&step, &g, cyclic ? k : 2 * k + 1, &Q);
    bn_set_u64(&pw, 1);
    bn_set_u64(&acc, 0);
    for (size_t j = 0; j < N; ++j) {
        load_elem(&xe, x, j, width);
        mod_mul(&term, &xe, &pw, &Q);
        mod_add(&acc, &acc, &term, &Q);
        mod_mul(&pw, &pw, &step, &Q);
    }
    store_elem(out, 0, &acc, width);
    return 0;
}

/*
 * One output of the inverse transform from the definition, O(N):
 *   cyclic:      x_j = N^{-1} sum_k y_k w^{-jk}
 *   negacyclic:  x_j = N^{-1} sum_k y_k psi^{-(2k+1) j}
 * `y` in natural order; `j` the coefficient index.
 */
int oracle_intt_point(uint64_t *out, const uint64_t *y, unsigned log2n, const uint64_t *q,
                      const uint64_t *root, int width, unsigned flags, uint64_t j) {
    if (check_args(q, width) || log2n > 30) return -1;
    size_t N = (size_t)1 << log2n;
    if (j >= N) return -1;
    int cyclic = (flags & OR_CYCLIC) != 0;
    bn Q, g, gi, step, base, pw, acc, ye, term, N_bn, ninv;
    bn_set_words(&Q, q, arg_words(width));
    bn_set_words(&g, root, arg_words(width));
    mod_inv(&gi, &g, &Q);
    /* term k uses gi^{jk} (cyclic) or gi^{(2k+1)j} = gi^j * (gi^{2j})^k (negacyclic) */
    if (cyclic) {
        mod_pow_u64(&step, &gi, j, &Q);
        bn_set_u64(&base, 1);
    } else {
        mod_pow_u64(&step, &gi, 2 * j, &Q);
        mod_pow_u64(&base, &gi, j, &Q);
    }
    pw = base;
    bn_set_u64(&acc, 0);
    for (size_t k = 0; k < N; ++k) {
        load_elem(&ye, y, k, width);
        mod_mul(&term, &ye, &pw, &Q);
        mod_add(&acc, &acc, &term, &Q);
        mod_mul(&pw, &pw, &step, &Q);
    }
    bn_set_u64(&N_bn, (uint64_t)N);
    mod_inv(&ninv, &N_bn, &Q);
    mod_mul(&acc, &acc, &ninv, &Q);
    store_elem(out, 0, &acc, width);
    return 0;
}

/*
 * Negacyclic (mod x^N + 1) schoolbook product, the polynomial product of Sec. 2.3 folded by
 * x^N = -1:  c_k = sum_{i+j=k} a_i b_j - sum_{i+j=k+N} a_i b_j  mod q.
 * out must not alias a or b.
 * Pinned by: hand-computed small products, x^{N-1} * x = -1, commutativity, and the identity.
 */
int oracle_negacyclic_mul(uint64_t *out, const uint64_t *a, const uint64_t *b, unsigned log2n,
                          const uint64_t *q, int width) {
    if (check_args(q, width) || log2n > 14) return -1;
    size_t N = (size_t)1 << log2n;
    bn Q, acc, ai, bj, p;
    bn_set_words(&Q, q, arg_words(width));
    for (size_t k = 0; k < N; ++k) {
        bn_set_u64(&acc, 0);
        for (size_t i = 0; i < N; ++i) {
            load_elem(&ai, a, i, width);
            if (i <= k) { /* i + j = k */
                load_elem(&bj, b, k - i, width);
                mod_mul(&p, &ai, &bj, &Q);
                mod_add(&acc, &acc, &p, &Q);
            } else { /* i + j = k + N, j = k + N - i in [k+1, N-1] */
                load_elem(&bj, b, k + N - i, width);
                mod_mul(&p, &ai, &bj, &Q);
                mod_sub(&acc, &acc, &p, &Q);
            }
        }
        store_elem(out, k, &acc, width);
    }
    return 0;
}

/*
 * Modular exponentiation g^e mod q (square-and-multiply), exposed for the tests' checks of
 * generated roots.  e is two words, low first.
 */
int oracle_powmod(uint64_t *out, const uint64_t g[2], const uint64_t e[2], const uint64_t q[2]) {
    if (q[1] == 0 && q[0] < 2) return -1;
    bn G, E, Q, R;
    bn_set_words(&G, g, 2);
    bn_set_words(&E, e, 2);
    bn_set_words(&Q, q, 2);
    mod_pow(&R, &G, &E, &Q);
    bn_get_words(&R, out, 2);
    return 0;
}

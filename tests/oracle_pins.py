"""Pins for the CPU oracle: checks against what the paper and the mathematics fix, not against the
oracle itself.

Each ``pin_*`` function takes an ``oracle.Oracle`` instance and raises ``AssertionError`` when the
oracle disagrees with:
  * the worked example of Sec. 2.3 (tests/golden/toy_ntt_q5.txt),
  * Python's own big integers (``%``, ``pow``) on random and limb-boundary operands,
  * the O(N^2) definition of Eq. 11 (and its negacyclic reading) computed here with Python integers
    on tiny N,
  * closed forms (unit vectors, the all-ones vector), invariants (inverse(forward(x)) = x,
    linearity, the convolution theorem against the schoolbook product), field identities.
``test_oracle_pins.py`` runs them on the real oracle; ``test_oracle_mutants.py`` runs them on
copies of the oracle with a plausible mistake planted, and expects at least one to fail.
"""
from __future__ import annotations

import functools
import os
import random

import numpy as np

from paper_2509_12494_gb300 import workload as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
VADD, VSUB, VMUL, AXPY = 0, 1, 2, 3
CYCLIC, BITREV = 1, 2


# ------------------------------------------------------------------ independent Python references

def brv(i: int, bits: int) -> int:
    return int(format(i, f"0{bits}b")[::-1], 2) if bits else 0


def py_forward(x, q, root, cyclic):
    """Eq. 11 (cyclic) or its negacyclic reading, straight from the sum, with Python integers."""
    N = len(x)
    if cyclic:
        return [sum(x[j] * pow(root, j * k, q) for j in range(N)) % q for k in range(N)]
    return [sum(x[j] * pow(root, (2 * k + 1) * j, q) for j in range(N)) % q for k in range(N)]


def py_inverse(y, q, root, cyclic):
    N = len(y)
    ninv, rinv = pow(N, -1, q), pow(root, -1, q)
    if cyclic:
        return [ninv * sum(y[k] * pow(rinv, j * k, q) for k in range(N)) % q for j in range(N)]
    return [ninv * sum(y[k] * pow(rinv, (2 * k + 1) * j, q) for k in range(N)) % q for j in range(N)]


def py_negacyclic(a, b, q):
    """Schoolbook product of Sec. 2.3 folded by x^N = -1."""
    N = len(a)
    c = [0] * (2 * N)
    for i in range(N):
        for j in range(N):
            c[i + j] += a[i] * b[j]
    return [(c[k] - c[k + N]) % q for k in range(N)]


def to_bitrev(v):
    bits = (len(v) - 1).bit_length()
    return [v[brv(i, bits)] for i in range(len(v))]


# ------------------------------------------------------------------ fixtures

def _largest_prime(bits: int, m: int) -> int:
    k = (1 << (bits - m)) - 1
    while True:
        q = (k << m) + 1
        if q.bit_length() == bits and W.is_probable_prime(q):
            return q
        k -= 1


@functools.lru_cache(maxsize=None)
def moduli(max_width: int = 2):
    """(q, width, max log2 of a negacyclic size) for small, 60-bit, 64-bit and 124-bit primes, and
    for a build that takes them, 188-bit (three words) and 252-bit (four words) primes."""
    wide = [
        (W.gen_prime(188, 18, 15), 3, 12),
        (W.gen_prime(252, 18, 16), 4, 12),
        (_largest_prime(252, 18), 4, 12),
        (W.gen_prime(160, 18, 17), 3, 12),
    ] if max_width >= 4 else []
    return [
        (17, 1, 3),
        (97, 1, 4),
        (7681, 1, 8),
        (W.gen_prime(60, 18, 11), 1, 17),
        (_largest_prime(60, 18), 1, 17),
        (W.gen_prime(64, 18, 12), 1, 17),
        (W.gen_prime(124, 18, 13), 2, 17),
        (_largest_prime(124, 18), 2, 17),
        (W.gen_prime(90, 18, 14), 2, 17),
    ] + wide


def edge_operands(q: int):
    cands = [0, 1, 2, q - 1, q - 2, (q - 1) // 2, (q + 1) // 2, 2**32 - 1, 2**32, 2**63, 2**64 - 1, 2**64,
             2**64 + 1, 2**96 - 1, 2**96, 2**123, 2**128 - 1, 2**128, 2**160, 2**187, 2**192 - 1, 2**192, 2**224,
             2**251]
    return sorted({c for c in cands if 0 <= c < q})


def arr(vals, width):
    return W.from_ints(vals, width)


def ints(a):
    return W.to_ints(np.asarray(a))


def load_golden():
    d = {}
    with open(os.path.join(GOLDEN, "toy_ntt_q5.txt")) as f:
        for line in f:
            line = line.split("#")[0].split()
            if not line:
                continue
            if line[0] == "w":
                d.setdefault("cases", []).append((int(line[1]), [int(v) for v in line[3:]]))
            else:
                d[line[0]] = [int(v) for v in line[1:]]
    return d


# ------------------------------------------------------------------ pins

def pin_toy_example(O):
    """Sec. 2.3 worked example: f = x^3 + 3x^2 + 2x + 1 mod 5 to {f(1), f(2), f(3), f(4)}."""
    g = load_golden()
    q, log2n, x = g["q"][0], g["log2n"][0], g["x"]
    assert sorted(g["evaluations"]) == sorted(
        sum(c * pow(t, i, q) for i, c in enumerate(x)) % q for t in range(1, q))
    for w, y in g["cases"]:
        xa = np.array(x, dtype=np.uint64)
        assert ints(O.ntt(xa, log2n, q, w, 1, CYCLIC)) == y
        assert ints(O.dft(xa, log2n, q, w, 1, CYCLIC)) == y
        assert sorted(y) == sorted(g["evaluations"])
        assert ints(O.ntt(np.array(y, dtype=np.uint64), log2n, q, w, 1, CYCLIC, inverse=True)) == x
        assert ints(O.dft(np.array(y, dtype=np.uint64), log2n, q, w, 1, CYCLIC, inverse=True)) == x


def pin_blas_python_ints(O):
    """Each BLAS op against Python's exact integers on edge and random operands (Sec. 2.1, Eq. 1)."""
    rnd = random.Random(1)
    for q, width, _ in moduli(O.max_width):
        e = edge_operands(q)
        a = [x for x in e for _ in e] + [rnd.randrange(q) for _ in range(64)]
        b = [y for _ in e for y in e] + [rnd.randrange(q) for _ in range(64)]
        A, B = arr(a, width), arr(b, width)
        assert ints(O.blas(VADD, A, B, q, width)) == [(x + y) % q for x, y in zip(a, b)]
        assert ints(O.blas(VSUB, A, B, q, width)) == [(x - y) % q for x, y in zip(a, b)]
        assert ints(O.blas(VMUL, A, B, q, width)) == [(x * y) % q for x, y in zip(a, b)]
        for s in e[:4] + [rnd.randrange(q)]:
            assert ints(O.blas(AXPY, A, B, q, width, s=s)) == [(s * x + y) % q for x, y in zip(a, b)]


def pin_blas_identities(O):
    """Field identities of Z_q for the BLAS ops."""
    rnd = random.Random(2)
    for q, width, _ in moduli(O.max_width):
        n = 48
        a = [rnd.randrange(q) for _ in range(n)]
        b = [rnd.randrange(q) for _ in range(n)]
        c = [rnd.randrange(q) for _ in range(n)]
        A, B, C = arr(a, width), arr(b, width), arr(c, width)
        one, zero = arr([1] * n, width), arr([0] * n, width)
        add = lambda x, y: O.blas(VADD, x, y, q, width)
        sub = lambda x, y: O.blas(VSUB, x, y, q, width)
        mul = lambda x, y: O.blas(VMUL, x, y, q, width)
        assert ints(add(A, B)) == ints(add(B, A))
        assert ints(mul(A, B)) == ints(mul(B, A))
        assert ints(sub(add(A, B), B)) == a
        assert ints(sub(A, A)) == [0] * n
        assert ints(mul(A, one)) == a
        assert ints(mul(A, zero)) == [0] * n
        assert ints(mul(A, add(B, C))) == ints(add(mul(A, B), mul(A, C)))
        s = rnd.randrange(q)
        assert ints(O.blas(AXPY, A, B, q, width, s=s)) == ints(add(mul(arr([s] * n, width), A), B))
        assert ints(O.blas(AXPY, A, B, q, width, s=1)) == ints(add(A, B))
        assert ints(O.blas(AXPY, A, B, q, width, s=q - 1)) == ints(sub(B, A))
        qm1 = arr([q - 1], width)
        assert ints(mul(qm1, qm1)) == [1]


def _ntt_cases(O):
    rnd = random.Random(3)
    for q, width, maxlog in moduli(O.max_width):
        for log2n in range(1, min(maxlog, 5) + 1):
            for cyclic in (False, True):
                root = W.gen_root(q, log2n, seed=log2n, cyclic=cyclic)
                yield q, width, log2n, cyclic, root, rnd


def pin_ntt_bruteforce(O):
    """Fast oracle NTT (both kinds, both orders, both directions) against the O(N^2) sum."""
    for q, width, log2n, cyclic, root, rnd in _ntt_cases(O):
        N = 1 << log2n
        x = [rnd.randrange(q) for _ in range(N)]
        ref = py_forward(x, q, root, cyclic)
        fl = CYCLIC if cyclic else 0
        assert ints(O.ntt(arr(x, width), log2n, q, root, width, fl)) == ref
        assert ints(O.ntt(arr(x, width), log2n, q, root, width, fl | BITREV)) == to_bitrev(ref)
        y = [rnd.randrange(q) for _ in range(N)]
        iref = py_inverse(y, q, root, cyclic)
        assert ints(O.ntt(arr(y, width), log2n, q, root, width, fl, inverse=True)) == iref
        assert ints(O.ntt(arr(to_bitrev(y), width), log2n, q, root, width, fl | BITREV, inverse=True)) == iref


def pin_dft_bruteforce(O):
    """The oracle's O(N^2) routine against the same sum written with Python integers."""
    for q, width, log2n, cyclic, root, rnd in _ntt_cases(O):
        if log2n > 4:
            continue
        N = 1 << log2n
        x = [rnd.randrange(q) for _ in range(N)]
        fl = CYCLIC if cyclic else 0
        assert ints(O.dft(arr(x, width), log2n, q, root, width, fl)) == py_forward(x, q, root, cyclic)
        assert ints(O.dft(arr(x, width), log2n, q, root, width, fl | BITREV)) == to_bitrev(
            py_forward(x, q, root, cyclic))
        assert ints(O.dft(arr(x, width), log2n, q, root, width, fl, inverse=True)) == py_inverse(
            x, q, root, cyclic)


def pin_closed_forms(O):
    """Unit vectors and the all-ones vector, whose transforms have closed forms."""
    for q, width, maxlog in moduli(O.max_width):
        for log2n in sorted({min(maxlog, 3), min(maxlog, 6), min(maxlog, 10)}):
            N = 1 << log2n
            psi = W.gen_root(q, log2n, seed=7)
            w = W.gen_root(q, log2n, seed=8, cyclic=True)
            e0, e1, ones = [1] + [0] * (N - 1), [0, 1] + [0] * (N - 2), [1] * N
            fwd = lambda v, r, fl: ints(O.ntt(arr(v, width), log2n, q, r, width, fl))
            assert fwd(e0, psi, 0) == [1] * N
            assert fwd(e0, w, CYCLIC) == [1] * N
            assert fwd(e1, psi, 0) == [pow(psi, 2 * k + 1, q) for k in range(N)]
            assert fwd(e1, w, CYCLIC) == [pow(w, k, q) for k in range(N)]
            assert fwd(ones, w, CYCLIC) == [N % q] + [0] * (N - 1)
            # sum_j psi^{(2k+1)j} = (1 - psi^{(2k+1)N}) / (1 - psi^{2k+1}) = 2 / (1 - psi^{2k+1})
            assert fwd(ones, psi, 0) == [2 * pow(1 - pow(psi, 2 * k + 1, q), -1, q) % q for k in range(N)]
            assert ints(O.ntt(arr([1] * N, width), log2n, q, psi, width, 0, inverse=True)) == e0
            if log2n <= 6:
                assert ints(O.dft(arr(e1, width), log2n, q, psi, width, 0)) == [pow(psi, 2 * k + 1, q)
                                                                                 for k in range(N)]
                assert ints(O.dft(arr(ones, width), log2n, q, w, width, CYCLIC)) == [N % q] + [0] * (N - 1)


def pin_roundtrip_and_linearity(O):
    """inverse(forward(x)) = x in both orders; forward(a + c*b) = forward(a) + c*forward(b)."""
    rnd = random.Random(4)
    for q, width, maxlog in moduli(O.max_width):
        log2n = min(maxlog, 9)
        N = 1 << log2n
        psi = W.gen_root(q, log2n, seed=9)
        a = [rnd.randrange(q) for _ in range(N)]
        b = [rnd.randrange(q) for _ in range(N)]
        c = rnd.randrange(q)
        for fl in (0, BITREV):
            ya = O.ntt(arr(a, width), log2n, q, psi, width, fl)
            assert ints(O.ntt(ya, log2n, q, psi, width, fl, inverse=True)) == a
        ya, yb = ints(O.ntt(arr(a, width), log2n, q, psi, width)), ints(O.ntt(arr(b, width), log2n, q, psi, width))
        comb = [(x + c * y) % q for x, y in zip(a, b)]
        assert ints(O.ntt(arr(comb, width), log2n, q, psi, width)) == [(x + c * y) % q for x, y in zip(ya, yb)]


def pin_convolution(O):
    """Convolution theorem: inverse(forward(a) . forward(b)) = schoolbook product mod x^N + 1."""
    rnd = random.Random(5)
    for q, width, maxlog in moduli(O.max_width):
        for log2n in sorted({min(maxlog, 4), min(maxlog, 7)}):
            N = 1 << log2n
            psi = W.gen_root(q, log2n, seed=10)
            a = [rnd.randrange(q) for _ in range(N)]
            b = [rnd.randrange(q) for _ in range(N)]
            ref = py_negacyclic(a, b, q)
            assert ints(O.negacyclic_mul(arr(a, width), arr(b, width), log2n, q, width)) == ref
            ya = ints(O.ntt(arr(a, width), log2n, q, psi, width))
            yb = ints(O.ntt(arr(b, width), log2n, q, psi, width))
            prod = [(x * y) % q for x, y in zip(ya, yb)]
            assert ints(O.ntt(arr(prod, width), log2n, q, psi, width, inverse=True)) == ref


def pin_negacyclic_mul(O):
    """Hand-worked product, x^{N-1} * x = -1, identity and commutativity."""
    # (1 + 2x)(x^2 + x^3) = x^2 + 3x^3 + 2x^4 = -2 + x^2 + 3x^3 mod (x^4 + 1, 17)
    assert ints(O.negacyclic_mul(arr([1, 2, 0, 0], 1), arr([0, 0, 1, 1], 1), 2, 17, 1)) == [15, 0, 1, 3]
    rnd = random.Random(6)
    for q, width, maxlog in moduli(O.max_width):
        log2n = min(maxlog, 5)
        N = 1 << log2n
        top, x1 = [0] * (N - 1) + [1], [0, 1] + [0] * (N - 2)
        assert ints(O.negacyclic_mul(arr(top, width), arr(x1, width), log2n, q, width)) == [q - 1] + [0] * (N - 1)
        a = [rnd.randrange(q) for _ in range(N)]
        b = [rnd.randrange(q) for _ in range(N)]
        one = [1] + [0] * (N - 1)
        assert ints(O.negacyclic_mul(arr(a, width), arr(one, width), log2n, q, width)) == a
        assert ints(O.negacyclic_mul(arr(a, width), arr(b, width), log2n, q, width)) == ints(
            O.negacyclic_mul(arr(b, width), arr(a, width), log2n, q, width))


def pin_points(O):
    """Single-output routines against the Python sum (small N) and against the pinned fast NTT."""
    rnd = random.Random(7)
    for q, width, maxlog in moduli(O.max_width):
        log2n = min(maxlog, 5)
        N = 1 << log2n
        for cyclic in (False, True):
            root = W.gen_root(q, log2n, seed=12, cyclic=cyclic)
            fl = CYCLIC if cyclic else 0
            x = [rnd.randrange(q) for _ in range(N)]
            ref, iref = py_forward(x, q, root, cyclic), py_inverse(x, q, root, cyclic)
            for k in range(N):
                assert O.ntt_point(arr(x, width), log2n, q, root, width, k, fl) == ref[k]
                assert O.intt_point(arr(x, width), log2n, q, root, width, k, fl) == iref[k]
        if maxlog >= 12:
            log2n = 12
            psi = W.gen_root(q, log2n, seed=13)
            x = [rnd.randrange(q) for _ in range(1 << log2n)]
            y = ints(O.ntt(arr(x, width), log2n, q, psi, width))
            for k in (0, 1, 2047, 4095):
                assert O.ntt_point(arr(x, width), log2n, q, psi, width, k) == y[k]
                assert O.intt_point(arr(y, width), log2n, q, psi, width, k) == x[k]


def pin_batched_stride(O):
    """A batch with a stride larger than N transforms each polynomial alone and skips the gaps."""
    for q, width, maxlog in moduli(O.max_width)[3:]:
        log2n, batch = 4, 3
        N = 1 << log2n
        stride = N + 5
        psi = W.gen_root(q, log2n, seed=14)
        flat = W.gen_residues(batch * stride, q, seed=15, width=width)
        x = flat.reshape((batch, stride) if width == 1 else (batch, stride, width)).copy()
        ref = [ints(O.ntt(x[b, :N].copy(), log2n, q, psi, width)) for b in range(batch)]
        xb = O.ntt_strided(flat, batch, stride, log2n, q, psi, width).reshape(x.shape)
        for b in range(batch):
            assert ints(xb[b, :N]) == ref[b]
            assert ints(xb[b, N:]) == ints(x[b, N:])


def pin_powmod(O):
    rnd = random.Random(8)
    for q, width, _ in moduli(O.max_width):
        if width > 2:
            continue  # oracle_powmod takes two-word operands
        for _ in range(8):
            g, e = rnd.randrange(q), rnd.randrange(2**128)
            assert O.powmod(g, e, q) == pow(g, e, q)


PINS = [pin_toy_example, pin_blas_python_ints, pin_blas_identities, pin_ntt_bruteforce, pin_dft_bruteforce,
        pin_closed_forms, pin_roundtrip_and_linearity, pin_convolution, pin_negacyclic_mul, pin_points,
        pin_batched_stride, pin_powmod]

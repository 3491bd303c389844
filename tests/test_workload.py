"""The seeded input generators: primes, roots of unity and residue vectors."""
import random

import numpy as np
import pytest

from paper_2509_12494_gb300 import workload as W

KNOWN_PRIMES = [2, 3, 5, 7681, 12289, 2**31 - 1, 2**61 - 1, 2**89 - 1, 2**107 - 1, 2**127 - 1,
                0xFFFFFFFF00000001]  # the last is the "Goldilocks" prime 2^64 - 2^32 + 1
# Carmichael numbers and strong pseudoprimes to several small bases
KNOWN_COMPOSITES = [1, 4, 561, 1105, 41041, 825265, 321197185, 3215031751, 2152302898747,
                    3474749660383, 341550071728321, 3825123056546413051, (2**61 - 1) * (2**31 - 1),
                    (2**64 + 13) * (2**59 + 21)]


def test_miller_rabin_known_values():
    for p in KNOWN_PRIMES:
        assert W.is_probable_prime(p), p
    for c in KNOWN_COMPOSITES:
        assert not W.is_probable_prime(c), c


def test_miller_rabin_agrees_with_sympy():
    sympy = pytest.importorskip("sympy")
    rnd = random.Random(21)
    for bits in (20, 40, 60, 64, 90, 124):
        for _ in range(200):
            n = rnd.getrandbits(bits) | 1
            assert W.is_probable_prime(n) == sympy.isprime(n), n


@pytest.mark.parametrize("bits,m", [(60, 17), (60, 18), (124, 17), (124, 18), (64, 12), (30, 11)])
def test_gen_prime_properties(bits, m):
    for seed in range(3):
        q = W.gen_prime(bits, m, seed)
        assert q.bit_length() == bits
        assert q % (1 << m) == 1
        assert W.is_probable_prime(q)
        assert W.gen_prime(bits, m, seed) == q  # deterministic
    try:
        import sympy
        assert sympy.isprime(q)
    except ImportError:
        pass


@pytest.mark.parametrize("log2n", [1, 2, 5, 10, 16, 17])
def test_gen_root_order(log2n):
    q = W.gen_prime(124, 18, 3)
    N = 1 << log2n
    psi = W.gen_root(q, log2n, seed=1)
    assert pow(psi, N, q) == q - 1 and pow(psi, 2 * N, q) == 1
    w = W.gen_root(q, log2n, seed=1, cyclic=True)
    assert pow(w, N, q) == 1 and pow(w, N // 2, q) == q - 1
    with pytest.raises(ValueError):
        W.gen_root(97, 10, seed=0)  # 2048 does not divide 96


@pytest.mark.parametrize("bits,width", [(60, 1), (64, 1), (124, 2), (90, 2), (65, 2), (17, 1), (188, 3), (150, 3),
                                        (252, 4), (200, 4)])
def test_gen_residues_range_and_determinism(bits, width):
    q = W.gen_prime(bits, min(bits - 2, 10), 5)
    a = W.gen_residues(10000, q, seed=9, width=width)
    b = W.gen_residues(10000, q, seed=9, width=width)
    assert np.array_equal(a, b)
    assert a.shape == ((10000,) if width == 1 else (10000, width))
    vals = W.to_ints(a)
    assert max(vals) < q and min(vals) >= 0
    # roughly uniform: the mean of v/q is near 1/2 and both halves of [0, q) are hit
    mean = sum(v / q for v in vals) / len(vals)
    assert abs(mean - 0.5) < 0.02
    assert not np.array_equal(a, W.gen_residues(10000, q, seed=10, width=width))


def test_int_round_trip():
    vals = [0, 1, 2**64 - 1, 2**64, 2**124 - 3]
    assert W.to_ints(W.from_ints(vals, 2)) == vals
    wide = vals + [2**128, 2**191 + 5, 2**255 + 2**64 + 1]
    assert W.to_ints(W.from_ints(wide, 4)) == wide
    assert W.to_ints(W.from_ints(wide[:-1], 3)) == wide[:-1]
    assert W.to_ints(W.from_ints([0, 5, 2**64 - 1], 1)) == [0, 5, 2**64 - 1]

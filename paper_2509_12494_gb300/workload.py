"""Seeded synthetic inputs shared by the tests, the oracle checks and the benchmark.

This module draws moduli, roots of unity and residue vectors.  It holds none of the transform or
BLAS arithmetic: it only picks parameters (with Miller-Rabin and Python's built-in ``pow``) and
draws uniform integers.  Both the CUDA path and the CPU oracle consume what it produces.

Recipes (FHE-shaped, matching the workloads the library is measured on):
  * prime q = k * 2^m + 1 with exactly ``bits`` bits, k uniform in [2^(bits-1-m), 2^(bits-m));
    accepted when it passes trial division and Miller-Rabin with 64 seeded random bases;
  * root: g uniform in [2, q-1]; psi = g^((q-1)/(2N)); accepted when psi^N = q-1, which makes its
    order exactly 2N (2N is a power of two).  For the cyclic transform, w = psi^2 has order N;
  * residues uniform in [0, q) by rejection of ceil(log2 q)-bit draws from numpy's PCG64.
Arrays are numpy uint64: shape (n,) for 64-bit residues and (n, 2) -- low word first -- for
128-bit residues (the memory layout the library reads).
"""
from __future__ import annotations

import random

import numpy as np

_SMALL_PRIMES = [p for p in range(3, 2000) if all(p % d for d in range(2, int(p**0.5) + 1))]


def is_probable_prime(n: int, rounds: int = 64, seed: int = 0x5EED) -> bool:
    """Trial division by small primes, then Miller-Rabin with `rounds` seeded random bases."""
    if n < 2:
        return False
    if n in (2, 3):
        return True
    if n % 2 == 0:
        return False
    for p in _SMALL_PRIMES:
        if n == p:
            return True
        if n % p == 0:
            return False
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    rnd = random.Random(seed ^ n)
    for _ in range(rounds):
        a = rnd.randrange(2, n - 1)
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def gen_prime(bits: int, m: int, seed: int) -> int:
    """Seeded random prime q = k*2^m + 1 of exactly `bits` bits (so q = 1 mod 2^m)."""
    if not (m + 2 <= bits):
        raise ValueError("need bits >= m + 2")
    rnd = random.Random(("prime", bits, m, seed).__repr__())
    lo, hi = 1 << (bits - 1 - m), 1 << (bits - m)
    while True:
        k = rnd.randrange(lo, hi)
        q = (k << m) + 1
        if q.bit_length() == bits and is_probable_prime(q):
            return q


def gen_root(q: int, log2n: int, seed: int, cyclic: bool = False) -> int:
    """Seeded primitive 2N-th root psi (negacyclic) or N-th root w (cyclic) modulo prime q."""
    N = 1 << log2n
    order = N if cyclic else 2 * N
    if (q - 1) % order:
        raise ValueError("q - 1 is not divisible by the root order")
    rnd = random.Random(("root", q, log2n, cyclic, seed).__repr__())
    half = order // 2
    while True:
        g = rnd.randrange(2, q - 1)
        r = pow(g, (q - 1) // order, q)
        if half == 0:
            if r == 1:
                return 1
            continue
        if pow(r, half, q) == q - 1:
            return r


def gen_residues(n: int, q: int, seed: int, width: int | None = None) -> np.ndarray:
    """n residues uniform in [0, q) (numpy PCG64, rejection sampling on bitlen(q)-bit draws).
    Shape (n,) for width 1, (n, width) -- low word first -- otherwise."""
    width = width or (1 if q < 2**64 else 2)
    bits = q.bit_length()
    rng = np.random.Generator(np.random.PCG64(seed))
    if width > 2:
        if q >= 1 << (64 * width):
            raise ValueError("q too large for the width")
        qw = [np.uint64((q >> (64 * k)) & (2**64 - 1)) for k in range(width)]
        top = width - 1
        tbits = min(max(bits - 64 * top, 0), 64)
        tmask = np.uint64((1 << tbits) - 1) if tbits < 64 else np.uint64(2**64 - 1)
        out = np.zeros((n, width), dtype=np.uint64)
        todo = np.arange(n)
        while todo.size:
            draw = [rng.bit_generator.random_raw(todo.size).astype(np.uint64) for _ in range(width)]
            draw[top] &= tmask
            less = np.zeros(todo.size, dtype=bool)   # draw < q, decided from the top word down
            equal = np.ones(todo.size, dtype=bool)
            for k in range(top, -1, -1):
                less |= equal & (draw[k] < qw[k])
                equal &= draw[k] == qw[k]
            for k in range(width):
                out[todo[less], k] = draw[k][less]
            todo = todo[~less]
        return out
    if width == 1:
        if q >= 2**64:
            raise ValueError("q too large for width 1")
        mask = np.uint64((1 << bits) - 1) if bits < 64 else np.uint64(2**64 - 1)
        out = np.empty(n, dtype=np.uint64)
        todo = np.arange(n)
        while todo.size:
            draw = rng.bit_generator.random_raw(todo.size).astype(np.uint64) & mask
            ok = draw < np.uint64(q)
            out[todo[ok]] = draw[ok]
            todo = todo[~ok]
        return out
    qlo, qhi = np.uint64(q & (2**64 - 1)), np.uint64(q >> 64)
    hbits = max(bits - 64, 0)
    hmask = np.uint64((1 << hbits) - 1)
    out = np.empty((n, 2), dtype=np.uint64)
    todo = np.arange(n)
    while todo.size:
        lo = rng.bit_generator.random_raw(todo.size).astype(np.uint64)
        hi = rng.bit_generator.random_raw(todo.size).astype(np.uint64) & hmask
        if bits <= 64:
            lo &= np.uint64((1 << bits) - 1) if bits < 64 else np.uint64(2**64 - 1)
        ok = (hi < qhi) | ((hi == qhi) & (lo < qlo))
        out[todo[ok], 0] = lo[ok]
        out[todo[ok], 1] = hi[ok]
        todo = todo[~ok]
    return out


def to_ints(a: np.ndarray) -> list[int]:
    """Residue array -> Python ints (for checks on small arrays); the last axis holds the words of
    a residue unless the array is one-dimensional (width 1)."""
    if a.ndim == 1:
        return [int(v) for v in a]
    w = a.shape[-1]
    return [sum(int(x) << (64 * k) for k, x in enumerate(r)) for r in a.reshape(-1, w)]


def from_ints(vals, width: int) -> np.ndarray:
    vals = [int(v) for v in vals]
    if width == 1:
        return np.array(vals, dtype=np.uint64)
    return np.array([[(v >> (64 * k)) & (2**64 - 1) for k in range(width)] for v in vals],
                    dtype=np.uint64).reshape(-1, width)


def words(v: int, n: int = 2) -> tuple[int, ...]:
    """A residue or modulus as n 64-bit words, low word first."""
    return tuple((v >> (64 * k)) & (2**64 - 1) for k in range(n))

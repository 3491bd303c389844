"""Helpers shared by the GPU parity tests."""
import numpy as np

from paper_2509_12494_gb300 import workload as W


def moduli():
    """(name, q, width): the widths' extremes and typical FHE-sized primes (all q = 1 mod 2^18)."""
    from tests.oracle_pins import _largest_prime
    return [
        ("q60", W.gen_prime(60, 18, 101), 1),
        ("q60max", _largest_prime(60, 18), 1),
        ("q40", W.gen_prime(40, 18, 102), 1),
        ("q124", W.gen_prime(124, 18, 103), 2),
        ("q124max", _largest_prime(124, 18), 2),
        ("q90", W.gen_prime(90, 18, 104), 2),
    ]


def sample_idx(n, k, seed):
    """k sorted distinct indices in [0, n) including both ends."""
    rng = np.random.default_rng(seed)
    idx = set(rng.choice(n, size=min(k, n), replace=False).tolist()) | {0, n - 1}
    return np.array(sorted(idx), dtype=np.int64)

"""The lazy butterflies at the edge of their bounds: the largest primes of each width (q just below
2^60 and 2^124, so 16q is just below the word) with inputs at q - 1, at 0 and mixed, through
one-pass and two-pass transforms, the batched form and the fused product, against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2509_12494_gb300 import workload as W
from tests.oracle_pins import _largest_prime

pytestmark = pytest.mark.gpu

QMAX = {1: _largest_prime(60, 18), 2: _largest_prime(124, 18)}


def _inputs(kind, n, q, width, seed):
    if kind == "max":
        return W.from_ints([q - 1] * n, width)
    if kind == "mixed":   # alternating q - 1 and 0, then random, so sums and differences hit both ends
        rnd = np.random.default_rng(seed)
        vals = [(q - 1) if (i % 3) else 0 for i in range(n)]
        for i in rnd.choice(n, size=n // 4, replace=False):
            vals[int(i)] = int(rnd.integers(0, 2**62)) % q
        return W.from_ints(vals, width)
    return W.gen_residues(n, q, seed=seed, width=width)


@pytest.mark.parametrize("kind", ["max", "mixed", "random"])
@pytest.mark.parametrize("width", [1, 2])
@pytest.mark.parametrize("log2n", [10, 13, 15])
@pytest.mark.parametrize("flags", [0, 2])
def test_largest_prime_transforms(mq, pool, log2n, width, kind, flags):
    import torch
    q = QMAX[width]
    psi = W.gen_root(q, log2n, seed=5)
    N = 1 << log2n
    x = _inputs(kind, N, q, width, log2n)
    plan = mq.ntt_plan_create(log2n, q, psi, width, flags)
    ofl = oracle.BITREV if flags & 2 else 0
    want_f = pool.submit(oracle.ntt, x.copy(), log2n, q, psi, width, ofl)
    want_i = pool.submit(oracle.ntt, x.copy(), log2n, q, psi, width, ofl, True)
    d = mq.to_device(x)
    mq.ntt_forward(plan, d)
    torch.cuda.synchronize()
    assert np.array_equal(mq.to_host(d), want_f.result())
    d = mq.to_device(x)
    mq.ntt_inverse(plan, d)
    torch.cuda.synchronize()
    assert np.array_equal(mq.to_host(d), want_i.result())


@pytest.mark.parametrize("width", [1, 2])
def test_largest_prime_batched_chain_and_product(mq, width):
    """Forward then inverse in one persistent launch, and the fused product, with inputs at q - 1."""
    import torch
    q = QMAX[width]
    log2n = 14
    N = 1 << log2n
    psi = W.gen_root(q, log2n, seed=6)
    plan = mq.ntt_plan_create(log2n, q, psi, width, mq.MQ_ORDER_BITREV)
    x = _inputs("max", 2 * N, q, width, 1)
    d = mq.to_device(x)
    jobs = [mq.ntt_job(mq.MQ_JOB_NTT_FORWARD, plan, d, 2, N),
            mq.ntt_job(mq.MQ_JOB_NTT_INVERSE, plan, d, 2, N, after=0)]
    b = mq.mq_batch_create(jobs)
    mq.mq_batch_launch(b)
    assert mq.mq_batch_status(b) == 0
    assert np.array_equal(mq.to_host(d), x)
    mq.mq_batch_destroy(b)
    a = _inputs("max", N, q, width, 2)
    c = _inputs("mixed", N, q, width, 3)
    dc = torch.empty_like(mq.to_device(a))
    mq.ntt_polymul(plan, dc, mq.to_device(a), mq.to_device(c))
    torch.cuda.synchronize()
    ref = oracle.ntt(oracle.blas(oracle.VMUL, oracle.ntt(a, log2n, q, psi, width),
                                 oracle.ntt(c, log2n, q, psi, width), q, width), log2n, q, psi, width, 0, True)
    assert np.array_equal(mq.to_host(dc), ref)

"""Whole polynomials at the largest sizes of the workloads, element by element against the oracle's
textbook transform (no sampling): N = 2^17 for every residue width, output order and direction, and
a polynomial of N = 2^16 taken from the 256-job batched form, in the batch the benchmark times."""
import numpy as np
import pytest

import oracle
from paper_2509_12494_gb300 import workload as W

pytestmark = pytest.mark.gpu


def _ofl(flags):
    return oracle.BITREV if flags & 2 else 0


@pytest.mark.parametrize("bits,width", [(60, 1), (124, 2)])
def test_whole_polynomials_2p17(mq, pool, bits, width):
    """For both orders and both directions: two polynomials of a batch of three (first and last),
    every output against oracle.ntt.  The inverse runs on independent random spectra."""
    import torch
    log2n, batch = 17, 3
    N = 1 << log2n
    q = W.gen_prime(bits, 18, 401)
    psi = W.gen_root(q, log2n, 401)
    shp = (batch, N) if width == 1 else (batch, N, width)
    x = W.gen_residues(batch * N, q, seed=402, width=width)
    xs = x.reshape(shp)
    jobs = []
    for flags in (0, 2):
        plan = mq.ntt_plan_create(log2n, q, psi, width, flags)
        for inverse in (False, True):
            d = mq.to_device(x)
            (mq.ntt_inverse if inverse else mq.ntt_forward)(plan, d, batch, N)
            torch.cuda.synchronize()
            got = mq.to_host(d).reshape(shp)
            for b in (0, batch - 1):
                f = pool.submit(oracle.ntt, xs[b].copy(), log2n, q, psi, width, _ofl(flags), inverse)
                jobs.append((flags, inverse, b, got[b].copy(), f))
    for flags, inverse, b, got, f in jobs:
        assert np.array_equal(got, f.result()), f"flags {flags}, inverse {inverse}, polynomial {b}"


@pytest.mark.parametrize("form", ["prefetch", "split"])
def test_whole_polynomial_from_the_uniform_batch(mq, pool, form):
    """The benchmark's batch (256 forward jobs of 2^16 under a 124-bit q = 1 mod 2^17, bit-reversed,
    then each inverse after its forward) with the inverse jobs left out, so that the forward results
    stay: three whole polynomials against oracle.ntt; then the full batch restores the input."""
    import torch
    log2n, batch = 16, 256
    N = 1 << log2n
    q = W.gen_prime(124, 17, 1)
    psi = W.gen_root(q, log2n, 1)
    plan = mq.ntt_plan_create(log2n, q, psi, 2, 2)
    x = W.gen_residues(batch * N, q, seed=11, width=2)
    flags = {"split": mq.MQ_BATCH_FORM_SPLIT, "prefetch": mq.MQ_BATCH_FORM_PREFETCH}[form]
    opts = mq.mq_batch_opts(flags=flags)
    d = mq.to_device(x)
    fwd = [mq.ntt_job(mq.MQ_JOB_NTT_FORWARD, plan, d[b * N:(b + 1) * N], 1, N) for b in range(batch)]
    fb = mq.mq_batch_create(fwd, opts)
    mq.mq_batch_launch(fb)
    assert mq.mq_batch_status(fb) == 0
    got = mq.to_host(d).reshape(batch, N, 2)
    xs = x.reshape(batch, N, 2)
    futs = [(b, pool.submit(oracle.ntt, xs[b].copy(), log2n, q, psi, 2, oracle.BITREV)) for b in (0, 131, 255)]
    for b, f in futs:
        assert np.array_equal(got[b], f.result()), f"polynomial {b}"
    d2 = mq.to_device(x)
    jobs = [mq.ntt_job(mq.MQ_JOB_NTT_FORWARD, plan, d2[b * N:(b + 1) * N], 1, N) for b in range(batch)]
    jobs += [mq.ntt_job(mq.MQ_JOB_NTT_INVERSE, plan, d2[b * N:(b + 1) * N], 1, N, after=b) for b in range(batch)]
    full = mq.mq_batch_create(jobs, opts)
    mq.mq_batch_launch(full)
    assert mq.mq_batch_status(full) == 0
    torch.cuda.synchronize()
    assert np.array_equal(mq.to_host(d2), x)

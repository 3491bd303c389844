"""The TMA forms of the 128-bit passes of tiles of 2^8 (N = 2^16 = 2^8 x 2^8, and the 2^8 side of
N = 2^15), element by element against the oracle's textbook transform.

The cases are those the copy engine must get right: polynomials stored with gaps between them
(stride N + 64; the gaps must come back untouched), an odd number of polynomials, both output
orders (the natural order's column pass takes the TMA form, its permuted row pass does not), both
directions, the per-call entry points and the batched form.  In the batch, TMA items run beside
items of the cp.async form: a 2^15 transform (column pass 2^7, cp.async; row pass 2^8, TMA) and a
60-bit transform."""
import numpy as np
import pytest

import oracle
from paper_2509_12494_gb300 import workload as W

pytestmark = pytest.mark.gpu

LOG2N, N = 16, 1 << 16
STRIDE = N + 64
BATCH = 19            # 19 x 2^8 tiles per pass = 608 groups of 8: the persistent TMA grid, not the latency shape
CHECK = (0, 9, 18)    # polynomials compared whole against the oracle


def _sync():
    import torch
    torch.cuda.synchronize()


def _ofl(flags):
    return oracle.BITREV if flags & 2 else 0


def _strided_input(q, seed, width=2, batch=BATCH, stride=STRIDE):
    """batch polynomials `stride` residues apart; the gaps hold random words too (they must stay)."""
    return W.gen_residues(batch * stride, q, seed, width)


def _poly(flat, b, n, stride=STRIDE):
    return flat[b * stride:b * stride + n]


@pytest.mark.parametrize("flags", [0, 2])
@pytest.mark.parametrize("inverse", [False, True])
def test_per_call_strided_batch(mq, pool, flags, inverse):
    q = W.gen_prime(124, 18, 611)
    psi = W.gen_root(q, LOG2N, 611)
    plan = mq.ntt_plan_create(LOG2N, q, psi, 2, flags)
    flat = _strided_input(q, 612 + flags + inverse)
    d = mq.to_device(flat)
    (mq.ntt_inverse if inverse else mq.ntt_forward)(plan, d, BATCH, STRIDE)
    _sync()
    got = mq.to_host(d)
    futs = {b: pool.submit(oracle.ntt, _poly(flat, b, N).copy(), LOG2N, q, psi, 2, _ofl(flags), inverse)
            for b in CHECK}
    for b in range(BATCH):   # gaps untouched
        assert np.array_equal(got[b * STRIDE + N:(b + 1) * STRIDE], flat[b * STRIDE + N:(b + 1) * STRIDE]), b
    for b, f in futs.items():
        assert np.array_equal(_poly(got, b, N), f.result()), (flags, inverse, b)


@pytest.mark.parametrize("form", ["prefetch", "split", "calls"])
def test_batched_tma_items_beside_cp_async_items(mq, pool, form):
    """Forward then inverse (dependent jobs) of a strided 2^16 batch, with a 2^15 and a 60-bit
    transform in the same batch: every result equals the per-call path's, the round trip restores
    the input with the gaps untouched, and three whole 2^16 spectra equal the oracle's."""
    q = W.gen_prime(124, 18, 621)
    psi = W.gen_root(q, LOG2N, 621)
    plan = mq.ntt_plan_create(LOG2N, q, psi, 2, 2)
    flat = _strided_input(q, 622)
    d = mq.to_device(flat)
    spec = mq.to_device(flat)                      # forward alone, for the oracle comparison
    mq.ntt_forward(plan, spec, BATCH, STRIDE)

    q15 = W.gen_prime(124, 18, 623)
    p15 = mq.ntt_plan_create(15, q15, W.gen_root(q15, 15, 623), 2, 2)
    x15 = W.gen_residues(6 << 15, q15, 624, 2)
    d15, r15 = mq.to_device(x15), mq.to_device(x15)
    mq.ntt_forward(p15, r15, 6, 1 << 15)

    q60 = W.gen_prime(60, 18, 625)
    p60 = mq.ntt_plan_create(LOG2N, q60, W.gen_root(q60, LOG2N, 625), 1, 0)
    x60 = W.gen_residues(5 * N, q60, 626, 1)
    d60, r60 = mq.to_device(x60), mq.to_device(x60)
    mq.ntt_forward(p60, r60, 5, N)
    _sync()

    flag = {"prefetch": mq.MQ_BATCH_FORM_PREFETCH, "split": mq.MQ_BATCH_FORM_SPLIT, "calls": mq.MQ_BATCH_FORM_CALLS}[form]
    jobs = [mq.ntt_job(mq.MQ_JOB_NTT_FORWARD, plan, d, BATCH, STRIDE),
            mq.ntt_job(mq.MQ_JOB_NTT_FORWARD, p15, d15, 6, 1 << 15),
            mq.ntt_job(mq.MQ_JOB_NTT_FORWARD, p60, d60, 5, N)]
    b = mq.mq_batch_create(jobs, mq.mq_batch_opts(flags=flag))
    mq.mq_batch_launch(b)
    assert mq.mq_batch_status(b) == 0, mq.mq_last_error()
    _sync()
    assert np.array_equal(mq.to_host(d), mq.to_host(spec))
    assert np.array_equal(mq.to_host(d15), mq.to_host(r15))
    assert np.array_equal(mq.to_host(d60), mq.to_host(r60))
    got = mq.to_host(d)
    futs = {k: pool.submit(oracle.ntt, _poly(flat, k, N).copy(), LOG2N, q, psi, 2, oracle.BITREV, False) for k in CHECK}
    for k, f in futs.items():
        assert np.array_equal(_poly(got, k, N), f.result()), k

    # the inverse as a job that waits for a forward in the same batch: the input comes back
    d2 = mq.to_device(flat)
    jobs = [mq.ntt_job(mq.MQ_JOB_NTT_FORWARD, plan, d2, BATCH, STRIDE),
            mq.ntt_job(mq.MQ_JOB_NTT_INVERSE, plan, d2, BATCH, STRIDE, after=0)]
    b2 = mq.mq_batch_create(jobs, mq.mq_batch_opts(flags=flag))
    mq.mq_batch_launch(b2)
    assert mq.mq_batch_status(b2) == 0, mq.mq_last_error()
    _sync()
    assert np.array_equal(mq.to_host(d2), flat)

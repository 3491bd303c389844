"""MQ_CHECK_INPUTS: the input range check of the canonical-operand precondition (Sec. 2.1,
0 <= a, b < q).  Inputs are built on the CPU with one planted non-canonical residue (q itself, or
the largest value the residue's words hold); a checked call must return MQ_ERR_RANGE and leave every
output untouched, and on canonical inputs a checked call must equal the unchecked one."""
import numpy as np
import pytest

from paper_2509_12494_gb300 import workload as W

pytestmark = pytest.mark.gpu

CASES = [(60, 1), (124, 2)]


def _planted(x, width, pos, value):
    """Copy of residues x (shape (n,) or (n, width)) with residue `pos` replaced by `value`."""
    y = x.copy()
    if width == 1:
        y[pos] = np.uint64(value)
    else:
        y[pos] = [np.uint64((value >> (64 * k)) & (2**64 - 1)) for k in range(width)]
    return y


def _bad_values(q, width):
    """q itself, the largest value below the width's modulus bound (2^60 - 1, 2^124 - 1, 2^188 - 1,
    2^252 - 1: at least q), and the largest value the residue's words hold."""
    bound = {1: 60, 2: 124, 3: 188, 4: 252}[width]
    return [q, (1 << bound) - 1, (1 << (64 * width)) - 1]


def _sync():
    import torch
    torch.cuda.synchronize()


@pytest.mark.parametrize("bits,width", CASES)
@pytest.mark.parametrize("log2n,flags", [(10, 0), (14, 0), (14, 2)])
@pytest.mark.parametrize("inverse", [False, True])
def test_checked_transform_refuses_planted_residue(mq, bits, width, log2n, flags, inverse):
    q = W.gen_prime(bits, log2n + 1, 31)
    psi = W.gen_root(q, log2n, 31)
    N, batch = 1 << log2n, 3
    plan = mq.ntt_plan_create(log2n, q, psi, width, flags | mq.MQ_CHECK_INPUTS)
    x = W.gen_residues(batch * N, q, seed=5, width=width)
    call = mq.ntt_inverse if inverse else mq.ntt_forward
    for k, bad in enumerate(_bad_values(q, width)):
        pos = [0, batch * N - 1, N + 17][k]
        y = _planted(x, width, pos, bad)
        d = mq.to_device(y)
        with pytest.raises(mq.MqError) as e:
            call(plan, d, batch, N)
        assert e.value.code == mq.MQ_ERR_RANGE
        assert "d_data" in mq.mq_last_error()
        _sync()
        assert np.array_equal(mq.to_host(d), y), "a refused call changed its data"
    # canonical inputs: the checked plan gives the unchecked plan's result
    ref = mq.ntt_plan_create(log2n, q, psi, width, flags)
    d1, d2 = mq.to_device(x), mq.to_device(x)
    call(plan, d1, batch, N)
    call(ref, d2, batch, N)
    _sync()
    assert np.array_equal(mq.to_host(d1), mq.to_host(d2))


def test_checked_transform_ignores_stride_padding(mq):
    """Only the N residues of each polynomial are read, so padding between them may hold anything."""
    import torch
    log2n, batch = 13, 2
    q = W.gen_prime(124, log2n + 1, 32)
    psi = W.gen_root(q, log2n, 32)
    N, stride = 1 << log2n, (1 << log2n) + 8
    plan = mq.ntt_plan_create(log2n, q, psi, 2, mq.MQ_CHECK_INPUTS)
    ref = mq.ntt_plan_create(log2n, q, psi, 2, 0)
    host = np.full((batch * stride, 2), np.uint64(2**64 - 1), dtype=np.uint64)
    x = W.gen_residues(batch * N, q, seed=6, width=2)
    for b in range(batch):
        host[b * stride:b * stride + N] = x[b * N:(b + 1) * N]
    d1, d2 = mq.to_device(host), mq.to_device(host)
    mq.ntt_forward(plan, d1, batch, stride)
    mq.ntt_forward(ref, d2, batch, stride)
    torch.cuda.synchronize()
    assert np.array_equal(mq.to_host(d1), mq.to_host(d2))


@pytest.mark.parametrize("bits,width", CASES)
def test_checked_polymul_refuses_either_operand(mq, bits, width):
    log2n, batch = 13, 2
    q = W.gen_prime(bits, log2n + 1, 33)
    psi = W.gen_root(q, log2n, 33)
    N = 1 << log2n
    plan = mq.ntt_plan_create(log2n, q, psi, width, mq.MQ_CHECK_INPUTS)
    a = W.gen_residues(batch * N, q, seed=7, width=width)
    b = W.gen_residues(batch * N, q, seed=8, width=width)
    marker = np.full_like(a, np.uint64(0x5A5A5A5A5A5A5A5A))
    for which in ("d_a", "d_b"):
        aa = _planted(a, width, 5, q) if which == "d_a" else a
        bb = _planted(b, width, N + 3, q) if which == "d_b" else b
        da, db, dc = mq.to_device(aa), mq.to_device(bb), mq.to_device(marker)
        with pytest.raises(mq.MqError) as e:
            mq.ntt_polymul(plan, dc, da, db, batch, N)
        assert e.value.code == mq.MQ_ERR_RANGE and which in mq.mq_last_error()
        _sync()
        assert np.array_equal(mq.to_host(dc), marker)
    ref = mq.ntt_plan_create(log2n, q, psi, width, 0)
    da, db, c1, c2 = mq.to_device(a), mq.to_device(b), mq.to_device(marker), mq.to_device(marker)
    mq.ntt_polymul(plan, c1, da, db, batch, N)
    mq.ntt_polymul(ref, c2, da, db, batch, N)
    _sync()
    assert np.array_equal(mq.to_host(c1), mq.to_host(c2))


@pytest.mark.parametrize("bits,width", CASES + [(188, 3), (252, 4)])
@pytest.mark.parametrize("op", ["vadd", "vsub", "vmul", "axpy"])
def test_checked_blas_refuses_planted_residue(mq, bits, width, op):
    n = 4099
    q = W.gen_prime(bits, 18, 34)
    a = W.gen_residues(n, q, seed=9, width=width)
    b = W.gen_residues(n, q, seed=10, width=width)
    marker = np.full_like(a, np.uint64(0x5A5A5A5A5A5A5A5A))
    s = 12345 % q
    wf = width | mq.MQ_CHECK_INPUTS

    def run(da, db, dc, w):
        if op == "axpy":   # y = s x + y: x = a, y = c (in place)
            mq.mod_axpy(dc, s, da, n, q, w)
        else:
            getattr(mq, "mod_" + op)(dc, da, db, n, q, w)

    names = ("d_x", "d_y") if op == "axpy" else ("d_a", "d_b")
    for k, bad in enumerate(_bad_values(q, width)):
        which = k % 2
        aa = _planted(a, width, n - 1, bad) if which == 0 else a
        bb = _planted(b, width, 1000, bad) if which == 1 else b
        # axpy reads y (the output) as its second input
        da, db = mq.to_device(aa), mq.to_device(bb)
        dc = mq.to_device(bb) if op == "axpy" else mq.to_device(marker)
        before = mq.to_host(dc)
        with pytest.raises(mq.MqError) as e:
            run(da, db, dc, wf)
        assert e.value.code == mq.MQ_ERR_RANGE and names[which] in mq.mq_last_error()
        _sync()
        assert np.array_equal(mq.to_host(dc), before), "a refused call changed its output"
    da, db = mq.to_device(a), mq.to_device(b)
    c1 = mq.to_device(b) if op == "axpy" else mq.to_device(marker)
    c2 = mq.to_device(b) if op == "axpy" else mq.to_device(marker)
    run(da, db, c1, wf)
    run(da, db, c2, width)
    _sync()
    assert np.array_equal(mq.to_host(c1), mq.to_host(c2))


def test_checked_batch_runs_no_job_on_a_planted_residue(mq):
    """A batch with checked jobs: one planted residue stops every job (MQ_ERR_RANGE at
    mq_batch_status, every buffer untouched); after an update to canonical data the same batch
    runs and equals the per-call path."""
    log2n, N = 14, 1 << 14
    q = W.gen_prime(124, 18, 35)
    psi = W.gen_root(q, log2n, 35)
    plan_c = mq.ntt_plan_create(log2n, q, psi, 2, mq.MQ_CHECK_INPUTS | mq.MQ_ORDER_BITREV)
    plan = mq.ntt_plan_create(log2n, q, psi, 2, mq.MQ_ORDER_BITREV)
    q60 = W.gen_prime(60, 18, 36)
    x = W.gen_residues(2 * N, q, seed=11, width=2)
    u = W.gen_residues(N, q, seed=12, width=2)          # unchecked transform's data
    a = W.gen_residues(50000, q60, seed=13, width=1)
    b = W.gen_residues(50000, q60, seed=14, width=1)
    c0 = np.zeros_like(a)

    def jobs_of(dx, du, da, db, dc):
        return [mq.ntt_job(mq.MQ_JOB_NTT_FORWARD, plan_c, dx, 2, N),
                mq.ntt_job(mq.MQ_JOB_NTT_FORWARD, plan, du, 1, N),
                mq.blas_job(mq.MQ_JOB_VMUL, dc, da, db, 50000, q60, 1 | mq.MQ_CHECK_INPUTS)]

    xb = _planted(x, 2, N + 5, q)
    bb = _planted(b, 1, 49999, q60)
    for xx, aa, bbb in ((xb, a, b), (x, a, bb)):
        dx, du, da, db, dc = (mq.to_device(v) for v in (xx, u, aa, bbb, c0))
        batch = mq.mq_batch_create(jobs_of(dx, du, da, db, dc))
        mq.mq_batch_launch(batch)
        assert mq.mq_batch_status(batch) == mq.MQ_ERR_RANGE
        for dev, want in ((dx, xx), (du, u), (da, aa), (db, bbb), (dc, c0)):
            assert np.array_equal(mq.to_host(dev), want), "a job ran although the check failed"
    # the last batch again, with canonical data in new buffers
    dx, du, da, db, dc = (mq.to_device(v) for v in (x, u, a, b, c0))
    mq.mq_batch_update(batch, jobs_of(dx, du, da, db, dc))
    mq.mq_batch_launch(batch)
    assert mq.mq_batch_status(batch) == mq.MQ_OK
    rx, ru, rc = mq.to_device(x), mq.to_device(u), mq.to_device(c0)
    mq.ntt_forward(plan, rx, 2, N)
    mq.ntt_forward(plan, ru, 1, N)
    mq.mod_vmul(rc, mq.to_device(a), mq.to_device(b), 50000, q60, 1)
    _sync()
    for got, want in ((dx, rx), (du, ru), (dc, rc)):
        assert np.array_equal(mq.to_host(got), mq.to_host(want))


def test_server_and_noalloc_refuse_checked_work(mq):
    q = W.gen_prime(124, 18, 37)
    psi = W.gen_root(q, 12, 37)
    plan = mq.ntt_plan_create(12, q, psi, 2, mq.MQ_CHECK_INPUTS)
    d = mq.to_device(W.gen_residues(1 << 12, q, seed=15, width=2))
    with pytest.raises(mq.MqError) as e:
        mq.ntt_forward_noalloc(plan, d, 1, 1 << 12)
    assert e.value.code == mq.MQ_ERR_ARG
    srv = mq.mq_server_create(mq.mq_server_cfg())
    try:
        with pytest.raises(mq.MqError) as e:
            mq.mq_submit(srv, mq.ntt_job(mq.MQ_JOB_NTT_FORWARD, plan, d, 1, 1 << 12))
        assert e.value.code == mq.MQ_ERR_ARG
    finally:
        mq.mq_server_destroy(srv)

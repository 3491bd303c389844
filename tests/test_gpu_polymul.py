"""The fused polynomial product (ntt_polymul) against the oracle: the schoolbook negacyclic product
where it is affordable, the oracle's transforms composed with its pointwise product otherwise, and
sampled schoolbook coefficients at full size.  Bit-exact."""
import numpy as np
import pytest

import oracle
from paper_2509_12494_gb300 import workload as W
from tests.gpu_util import sample_idx

pytestmark = pytest.mark.gpu

Q = {1: W.gen_prime(60, 18, 501), 2: W.gen_prime(124, 18, 502)}


def _sync():
    import torch
    torch.cuda.synchronize()


def _polys(flat, batch, stride, width):
    return flat.reshape((batch, stride) if width == 1 else (batch, stride, 2))


def _schoolbook_coeff(a, b, k, q, cyclic=False):
    """Coefficient k of a * b mod (x^N + 1) (x^N - 1 if cyclic), from Python integers."""
    N = len(a)
    s = sum(a[i] * b[k - i] for i in range(k + 1))
    t = sum(a[i] * b[k + N - i] for i in range(k + 1, N))
    return (s + t if cyclic else s - t) % q


def _via_oracle_transforms(a, b, log2n, q, root, width, cyclic):
    """inverse(forward(a) * forward(b)) with the oracle's transform and pointwise product."""
    fl = oracle.CYCLIC if cyclic else 0
    A = oracle.ntt(a, log2n, q, root, width, fl)
    B = oracle.ntt(b, log2n, q, root, width, fl)
    return oracle.ntt(oracle.blas(oracle.VMUL, A, B, q, width), log2n, q, root, width, fl, True)


@pytest.mark.parametrize("width", [1, 2])
@pytest.mark.parametrize("log2n", list(range(1, 15)))
def test_negacyclic_product_vs_oracle(mq, pool, log2n, width):
    """Every size from 2 to 2^14 (the one-kernel form up to 2^12, the fused row pass above), a
    batch with a stride longer than N whose gaps stay untouched."""
    import torch
    q = Q[width]
    N = 1 << log2n
    root = W.gen_root(q, log2n, seed=log2n + 10 * width)
    plan = mq.ntt_plan_create(log2n, q, root, width, 0)
    batch = 3 if log2n <= 12 else 2
    stride = N + 5
    fa = W.gen_residues(batch * stride, q, seed=log2n * 3 + width, width=width)
    fb = W.gen_residues(batch * stride, q, seed=log2n * 5 + width, width=width)
    da, db = mq.to_device(fa), mq.to_device(fb)
    dc = mq.to_device(W.gen_residues(batch * stride, q, seed=99, width=width))  # junk, gaps kept
    gaps = _polys(mq.to_host(dc), batch, stride, width)[:, N:].copy()
    mq.ntt_polymul(plan, dc, da, db, batch, stride)
    _sync()
    got = _polys(mq.to_host(dc), batch, stride, width)
    A, B = _polys(fa, batch, stride, width), _polys(fb, batch, stride, width)
    if log2n <= 10:
        want = [pool.submit(oracle.negacyclic_mul, A[i, :N].copy(), B[i, :N].copy(), log2n, q, width)
                for i in range(batch)]
    else:
        want = [pool.submit(_via_oracle_transforms, A[i, :N].copy(), B[i, :N].copy(), log2n, q, root, width, False)
                for i in range(batch)]
    for i in range(batch):
        assert np.array_equal(got[i, :N], want[i].result()), (log2n, width, i)
    assert np.array_equal(got[:, N:], gaps), "gap written"
    assert np.array_equal(mq.to_host(da), fa) and np.array_equal(mq.to_host(db), fb), "inputs modified"
    torch.cuda.synchronize()


@pytest.mark.parametrize("log2n,width", [(9, 2), (12, 1), (13, 2), (14, 1)])
def test_cyclic_plan_gives_cyclic_product(mq, pool, log2n, width):
    q = Q[width]
    N = 1 << log2n
    root = W.gen_root(q, log2n, seed=7, cyclic=True)
    plan = mq.ntt_plan_create(log2n, q, root, width, mq.MQ_CYCLIC)
    a = W.gen_residues(N, q, seed=1, width=width)
    b = W.gen_residues(N, q, seed=2, width=width)
    dc = mq.to_device(a)
    mq.ntt_polymul(plan, dc, mq.to_device(a), mq.to_device(b))
    _sync()
    got = mq.to_host(dc)
    assert np.array_equal(got, _via_oracle_transforms(a, b, log2n, q, root, width, True))
    ai, bi = W.to_ints(a), W.to_ints(b)
    for k in sample_idx(N, 3, seed=log2n):
        assert W.to_ints(got[k:k + 1])[0] == _schoolbook_coeff(ai, bi, int(k), q, cyclic=True)


@pytest.mark.parametrize("alias", ["a", "b"])
@pytest.mark.parametrize("log2n", [11, 15])
def test_in_place(mq, log2n, alias):
    """c may be a or b: the result equals the out-of-place product."""
    import torch
    q = Q[2]
    N = 1 << log2n
    plan = mq.ntt_plan_create(log2n, q, W.gen_root(q, log2n, seed=3), 2, mq.MQ_ORDER_BITREV)
    a = W.gen_residues(2 * N, q, seed=11, width=2)
    b = W.gen_residues(2 * N, q, seed=12, width=2)
    da, db, dc = mq.to_device(a), mq.to_device(b), torch.empty(2 * N, 2, dtype=torch.int64, device="cuda")
    mq.ntt_polymul(plan, dc, da, db, 2, N)
    _sync()
    want = mq.to_host(dc)
    target = da if alias == "a" else db
    mq.ntt_polymul(plan, target, da, db, 2, N)
    _sync()
    assert np.array_equal(mq.to_host(target), want)


@pytest.mark.parametrize("log2n,width", [(16, 2), (17, 2), (16, 1)])
def test_full_size_sampled(mq, log2n, width):
    """FHE sizes (batch 4): sampled coefficients of the first and last product against the
    schoolbook sum, and the whole batch against the per-call path (forward, vmul, inverse), whose
    parity with the oracle the transform and BLAS tests establish."""
    import torch
    q = Q[width]
    N = 1 << log2n
    root = W.gen_root(q, log2n, seed=5)
    plan = mq.ntt_plan_create(log2n, q, root, width, mq.MQ_ORDER_BITREV)
    batch = 4
    a = W.gen_residues(batch * N, q, seed=21, width=width)
    b = W.gen_residues(batch * N, q, seed=22, width=width)
    da, db = mq.to_device(a), mq.to_device(b)
    dc = torch.empty_like(da)
    mq.ntt_polymul(plan, dc, da, db, batch, N)
    # the unfused composition on copies
    ta, tb = mq.to_device(a), mq.to_device(b)
    mq.ntt_forward(plan, ta, batch, N)
    mq.ntt_forward(plan, tb, batch, N)
    mq.mod_vmul(ta, ta, tb, batch * N, q, width)
    mq.ntt_inverse(plan, ta, batch, N)
    _sync()
    got = mq.to_host(dc)
    assert np.array_equal(got, mq.to_host(ta))
    P = _polys(got, batch, N, width)
    for i in (0, batch - 1):
        ai = W.to_ints(_polys(a, batch, N, width)[i])
        bi = W.to_ints(_polys(b, batch, N, width)[i])
        for k in sample_idx(N, 2, seed=i):
            assert W.to_ints(P[i, k:k + 1])[0] == _schoolbook_coeff(ai, bi, int(k), q), (log2n, i, int(k))


def test_edge_cases(mq):
    q = Q[2]
    plan = mq.ntt_plan_create(6, q, W.gen_root(q, 6, seed=1), 2, 0)
    mq.ntt_polymul(plan, None, None, None, 0)  # batch 0: no-op, pointers unused
    import torch
    d = torch.zeros(64, 2, dtype=torch.int64, device="cuda")
    with pytest.raises(mq.MqError) as e:
        mq.ntt_polymul(plan, d, d, d, 2, 63)   # stride below N
    assert e.value.code == mq.MQ_ERR_SIZE
    with pytest.raises(mq.MqError) as e:
        mq.ntt_polymul(plan, d.data_ptr() + 8, d, d)
    assert e.value.code == mq.MQ_ERR_ALIGN
    # x^(N-1) * x = x^N = -1 in the negacyclic ring
    x = np.zeros((64, 2), dtype=np.uint64)
    y = x.copy()
    x[63, 0] = 1
    y[1, 0] = 1
    dc = torch.empty(64, 2, dtype=torch.int64, device="cuda")
    mq.ntt_polymul(plan, dc, mq.to_device(x), mq.to_device(y))
    _sync()
    want = np.zeros((64, 2), dtype=np.uint64)
    want[0] = W.from_ints([q - 1], 2)[0]
    assert np.array_equal(mq.to_host(dc), want)

"""Residues of three and four 64-bit words (192- and 256-bit integers, the larger bit-widths of
Sec. 7): transforms and BLAS against the oracle's wide build, bit-exact."""
import numpy as np
import pytest

import oracle
from paper_2509_12494_gb300 import workload as W
from tests.gpu_util import sample_idx
from tests.oracle_pins import _largest_prime

pytestmark = pytest.mark.gpu

Q = {3: W.gen_prime(188, 18, 601), 4: W.gen_prime(252, 18, 602)}
QMAX = {3: _largest_prime(188, 18), 4: _largest_prime(252, 18)}
FLAGS = {"nega_nat": 0, "nega_brv": 2, "cyc_nat": 1, "cyc_brv": 3}


def _ofl(flags):
    return (oracle.CYCLIC if flags & 1 else 0) | (oracle.BITREV if flags & 2 else 0)


def _strided(flat, batch, stride, width):
    return flat.reshape(batch, stride, width)


@pytest.mark.parametrize("flag", list(FLAGS))
@pytest.mark.parametrize("width", [3, 4])
@pytest.mark.parametrize("log2n", [1, 2, 3, 5, 8, 10, 11, 12, 13, 14])
def test_wide_ntt_vs_oracle(mq, pool, log2n, width, flag):
    """One-pass (N <= 2^10) and two-pass sizes, both directions, both orders, both kinds; a batch
    whose stride is longer than N keeps its gaps."""
    import torch
    if log2n >= 12 and flag.startswith("cyc"):
        pytest.skip("cyclic checked up to 2^11 here")
    q = Q[width] if log2n % 2 else QMAX[width]
    flags = FLAGS[flag]
    root = W.gen_root(q, log2n, seed=log2n + width, cyclic=bool(flags & 1))
    N = 1 << log2n
    batch = 3 if log2n <= 10 else 2
    stride = N + 3
    flat = W.gen_residues(batch * stride, q, seed=log2n * 11 + width, width=width)
    plan = mq.ntt_plan_create(log2n, q, root, width, flags)
    for inverse in (False, True):
        d = mq.to_device(flat)
        (mq.ntt_inverse if inverse else mq.ntt_forward)(plan, d, batch, stride)
        torch.cuda.synchronize()
        got = _strided(mq.to_host(d), batch, stride, width)
        x = _strided(flat, batch, stride, width)
        futs = [pool.submit(oracle.ntt, x[b, :N].copy(), log2n, q, root, width, _ofl(flags), inverse)
                for b in range(batch)]
        for b in range(batch):
            assert np.array_equal(got[b, :N], futs[b].result()), (log2n, width, flag, inverse, b)
            assert np.array_equal(got[b, N:], x[b, N:]), "gap written"


@pytest.mark.parametrize("width", [3, 4])
@pytest.mark.parametrize("log2n", [16, 20])
def test_wide_large_sizes(mq, pool, log2n, width):
    """Large N: forward outputs at sampled points against the oracle's O(N) evaluation from the
    definition, and the round trip restores the input."""
    import torch
    q = W.gen_prime(188 if width == 3 else 252, 22, 603)  # q = 1 mod 2^22: roots of order up to 2^22
    psi = W.gen_root(q, log2n, seed=3)
    N = 1 << log2n
    x = W.gen_residues(N, q, seed=log2n + 7 * width, width=width)
    plan = mq.ntt_plan_create(log2n, q, psi, width, 0)
    d = mq.to_device(x)
    mq.ntt_forward(plan, d)
    torch.cuda.synchronize()
    y = mq.to_host(d)
    idx = sample_idx(N, 3 if log2n > 16 else 6, seed=width)
    futs = [(int(k), pool.submit(oracle.ntt_point, x, log2n, q, psi, width, int(k))) for k in idx]
    for k, f in futs:
        assert W.to_ints(y[k:k + 1])[0] == f.result(), (log2n, width, k)
    mq.ntt_inverse(plan, d)
    torch.cuda.synchronize()
    assert np.array_equal(mq.to_host(d), x)


@pytest.mark.parametrize("width", [3, 4])
@pytest.mark.parametrize("op", ["vadd", "vsub", "vmul", "axpy"])
def test_wide_blas_vs_oracle(mq, width, op):
    import torch
    for q in (Q[width], QMAX[width], W.gen_prime(64 * width - 40, 18, 9)):
        n = 9001
        a = W.gen_residues(n, q, seed=1, width=width)
        b = W.gen_residues(n, q, seed=2, width=width)
        edges = [0, 1, q - 1, q - 2, (q - 1) // 2, 2**64 - 1, 2**128 - 1]
        for i, v in enumerate(edges):
            if v < q:
                a[i] = W.from_ints([v], width)[0]
                b[-1 - i] = W.from_ints([v], width)[0]
        s = W.to_ints(W.gen_residues(1, q, seed=3, width=width))[0]
        da, db = mq.to_device(a), mq.to_device(b)
        if op == "axpy":
            mq.mod_axpy(db, s, da, n, q, width)
            want = oracle.blas(oracle.AXPY, a, b, q, width, s=s)
            got = db
        else:
            got = torch.empty_like(da)
            getattr(mq, "mod_" + op)(got, da, db, n, q, width)
            want = oracle.blas({"vadd": oracle.VADD, "vsub": oracle.VSUB, "vmul": oracle.VMUL}[op], a, b, q, width)
        torch.cuda.synchronize()
        assert np.array_equal(mq.to_host(got), want), (op, width, q.bit_length())


def test_wide_limits(mq):
    import torch
    q3 = Q[3]
    with pytest.raises(mq.MqError) as e:   # above the 188-bit bound of three words
        mq.ntt_plan_create(10, W.gen_prime(190, 18, 1), 3, 3, 0)
    assert e.value.code == mq.MQ_ERR_MODULUS
    with pytest.raises(mq.MqError) as e:   # transforms of wide residues stop at 2^20
        mq.ntt_plan_create(21, q3, W.gen_root(q3, 17, 1), 3, 0)
    assert e.value.code in (mq.MQ_ERR_SIZE, mq.MQ_ERR_MODULUS)
    plan = mq.ntt_plan_create(12, q3, W.gen_root(q3, 12, 1), 3, 0)
    d = torch.zeros(4096, 3, dtype=torch.int64, device="cuda")
    with pytest.raises(mq.MqError) as e:   # no fused product for wide residues
        mq.ntt_polymul(plan, d, d, d)
    assert e.value.code == mq.MQ_ERR_ARG
    with pytest.raises(mq.MqError) as e:   # nor batched jobs
        mq.mq_batch_create([mq.ntt_job(mq.MQ_JOB_NTT_FORWARD, plan, d, 1, 4096)])
    assert e.value.code == mq.MQ_ERR_ARG

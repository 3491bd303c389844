"""GPU modular BLAS vs the CPU oracle, element by element (bit-exact)."""
import numpy as np
import pytest

import oracle
from paper_2509_12494_gb300 import workload as W
from tests.gpu_util import moduli, sample_idx
from tests.oracle_pins import edge_operands

pytestmark = pytest.mark.gpu
OPS = {"vadd": oracle.VADD, "vsub": oracle.VSUB, "vmul": oracle.VMUL, "axpy": oracle.AXPY}


def run_gpu(M, op, a, b, q, width, s=0, out_alias=None):
    import torch
    n = a.shape[0]
    da, db = M.to_device(a), M.to_device(b)
    if op == "axpy":
        M.mod_axpy(db, s, da, n, q, width)
        res = db
    else:
        dc = da if out_alias == "a" else db if out_alias == "b" else torch.empty_like(da)
        getattr(M, "mod_" + op)(dc, da, db, n, q, width)
        res = dc
    torch.cuda.synchronize()
    return M.to_host(res)


@pytest.mark.parametrize("name,q,width", moduli(), ids=[m[0] for m in moduli()])
@pytest.mark.parametrize("op", list(OPS))
@pytest.mark.parametrize("n", [1, 2, 3, 255, 1024, 4099, 65537])
def test_blas_random(mq, op, name, q, width, n):
    a = W.gen_residues(n, q, seed=n, width=width)
    b = W.gen_residues(n, q, seed=n + 1, width=width)
    s = W.to_ints(W.gen_residues(1, q, seed=n + 2, width=width))[0]
    got = run_gpu(mq, op, a, b, q, width, s)
    assert np.array_equal(got, oracle.blas(OPS[op], a, b, q, width, s=s))


@pytest.mark.parametrize("name,q,width", moduli(), ids=[m[0] for m in moduli()])
@pytest.mark.parametrize("op", list(OPS))
def test_blas_edge_operands(mq, op, name, q, width):
    e = edge_operands(q)
    a = W.from_ints([x for x in e for _ in e], width)
    b = W.from_ints([y for _ in e for y in e], width)
    for s in e:
        got = run_gpu(mq, op, a, b, q, width, s)
        assert np.array_equal(got, oracle.blas(OPS[op], a, b, q, width, s=s)), s
        if op != "axpy":
            break


@pytest.mark.parametrize("op", ["vadd", "vsub", "vmul"])
@pytest.mark.parametrize("alias", ["a", "b"])
def test_blas_output_aliases_input(mq, op, alias):
    for _, q, width in moduli()[::3]:
        a = W.gen_residues(5000, q, seed=7, width=width)
        b = W.gen_residues(5000, q, seed=8, width=width)
        got = run_gpu(mq, op, a, b, q, width, out_alias=alias)
        assert np.array_equal(got, oracle.blas(OPS[op], a, b, q, width))


@pytest.mark.parametrize("op", list(OPS))
def test_blas_unaligned_64bit_vectors(mq, op):
    """64-bit residues at an 8-byte (not 16-byte) aligned start take the scalar path."""
    import torch
    _, q, width = moduli()[0]
    n = 1001
    a = W.gen_residues(n + 1, q, seed=1, width=1)
    b = W.gen_residues(n + 1, q, seed=2, width=1)
    da, db = mq.to_device(a), mq.to_device(b)
    dc = torch.zeros_like(da)
    if op == "axpy":
        mq.mod_axpy(db[1:], 12345, da[1:], n, q, 1)
        got = mq.to_host(db)[1:]
        ref = oracle.blas(oracle.AXPY, a[1:], b[1:], q, 1, s=12345)
    else:
        getattr(mq, "mod_" + op)(dc[1:], da[1:], db[1:], n, q, 1)
        got = mq.to_host(dc)[1:]
        ref = oracle.blas(OPS[op], a[1:], b[1:], q, 1)
    assert mq.to_host(dc)[0] == 0 or op == "axpy"
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("log2n", [20, 24])
@pytest.mark.parametrize("width", [1, 2])
@pytest.mark.parametrize("op", list(OPS))
def test_blas_full_size_sampled(mq, pool, op, width, log2n):
    """The benchmark's vector lengths: every element of a random sample against the oracle."""
    n = (1 << log2n) + (0 if log2n == 24 else 3)  # a ragged tail at 2^20
    q = W.gen_prime(60 if width == 1 else 124, 18, 200 + width)
    a = W.gen_residues(n, q, seed=log2n, width=width)
    b = W.gen_residues(n, q, seed=log2n + 1, width=width)
    s = W.to_ints(W.gen_residues(1, q, seed=5, width=width))[0]
    got = run_gpu(mq, op, a, b, q, width, s)
    idx = sample_idx(n, 20000, seed=log2n)
    assert np.array_equal(got[idx], oracle.blas(OPS[op], a[idx], b[idx], q, width, s=s))

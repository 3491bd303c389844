"""The two forms of the double-word product (Sec. 2.2: schoolbook, Eq. 8, and Karatsuba, Eq. 9)
inside the general 124-bit modular product: bit-exact against the oracle on random and edge
operands, and both measurable by the throughput probe."""
import numpy as np
import pytest

import oracle
from paper_2509_12494_gb300 import workload as W
from tests.gpu_util import moduli

pytestmark = pytest.mark.gpu

WIDE = [(name, q) for name, q, width in moduli() if width == 2]


def _edges(q, n, seed):
    """Random residues with the extremes planted: 0, 1, q - 1, q - 2, values with all-one halves."""
    x = W.gen_residues(n, q, seed, 2)
    special = [0, 1, q - 1, q - 2, (q - 1) // 2, (1 << 64) - 1, (1 << 123) - 1, ((1 << 64) - 1) << 58]
    for i, v in enumerate(special):
        if 0 <= v < q:
            x[i] = W.from_ints([v], 2)[0]
    return x


@pytest.mark.parametrize("name,q", WIDE)
@pytest.mark.parametrize("variant", ["schoolbook", "karatsuba"])
def test_product_forms_vs_oracle(mq, name, q, variant):
    import torch
    v = mq.MQ_MUL_KARATSUBA if variant == "karatsuba" else mq.MQ_MUL_SCHOOLBOOK
    n = 50021
    a = _edges(q, n, 3)
    b = _edges(q, n, 4)[::-1].copy()
    da, db = mq.to_device(a), mq.to_device(b)
    dc = torch.empty_like(da)
    mq.mq_probe_mulmod(v, dc, da, db, n, q)
    torch.cuda.synchronize()
    assert np.array_equal(mq.to_host(dc), oracle.blas(oracle.VMUL, a, b, q, 2)), (name, variant)


def test_rate_probe_reports_both(mq):
    q = W.gen_prime(124, 18, 7)
    r0, ms0 = mq.mq_probe_mulmod_rate(mq.MQ_MUL_SCHOOLBOOK, 64, q)
    r1, ms1 = mq.mq_probe_mulmod_rate(mq.MQ_MUL_KARATSUBA, 64, q)
    assert r0 > 1e9 and r1 > 1e9 and ms0 > 0 and ms1 > 0

"""ntt_forward_noalloc: the forward transform for callers that cannot allocate device memory while
running.  Its results must equal ntt_forward's bit for bit, call after call, although every call
reuses one static staging buffer.  This file is collected last so that a failing run that stops at
the first failure has already run every other test."""
import numpy as np
import pytest

from paper_2509_12494_gb300 import workload as W

pytestmark = pytest.mark.gpu


def _forward(M, fn, plan, x, batch, N):
    import torch
    d = M.to_device(x)
    fn(plan, d, batch, N)
    torch.cuda.synchronize()
    return M.to_host(d)


@pytest.mark.parametrize("bits,log2n,batch,flags", [
    (124, 16, 16, 0),   # natural order, two passes: stages through the static buffer (16 MiB, the limit)
    (60, 17, 8, 0),     # 8 MiB of staging for 64-bit residues
    (124, 13, 3, 0),    # smallest two-pass size
    (124, 10, 5, 0),    # one pass: no staging
    (124, 16, 64, 2),   # bit-reversed order: in place, no staging, any batch
])
def test_noalloc_matches_ntt_forward(mq, bits, log2n, batch, flags):
    width = 2 if bits > 60 else 1
    q = W.gen_prime(bits, log2n + 1, 7)
    psi = W.gen_root(q, log2n, 7)
    N = 1 << log2n
    plan = mq.ntt_plan_create(log2n, q, psi, width, flags)
    for call in range(2):  # two calls in a row: the second sees the first call's staging contents
        x = W.gen_residues(batch * N, q, seed=100 * call + log2n, width=width)
        want = _forward(mq, mq.ntt_forward, plan, x, batch, N)
        got = _forward(mq, mq.ntt_forward_noalloc, plan, x, batch, N)
        assert np.array_equal(got, want), f"call {call}"


def test_noalloc_rejects_batches_beyond_the_buffer(mq):
    import torch
    q = W.gen_prime(124, 17, 3)
    psi = W.gen_root(q, 16, 3)
    plan = mq.ntt_plan_create(16, q, psi, 2, 0)
    d = torch.zeros((17 << 16, 2), dtype=torch.int64, device="cuda")  # 17 MiB > 16 MiB of staging
    with pytest.raises(mq.MqError) as e:
        mq.ntt_forward_noalloc(plan, d, 17, 1 << 16)
    assert e.value.code == mq.MQ_ERR_SIZE
    assert "split the batch" in mq.mq_last_error()

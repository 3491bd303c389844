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


def _laid_out(mq, x, batch, N, stride, width, off_words):
    """A device buffer holding `batch` polynomials `stride` residues apart, starting `off_words`
    64-bit words into the allocation; every other word holds a marker.  Returns (buffer, view)."""
    import torch
    total = off_words + batch * stride * width + 8
    host = np.full(total, 0x5A5A5A5A5A5A5A5A, dtype=np.uint64)
    xs = x.reshape(batch, N * width)
    for b in range(batch):
        s = off_words + b * stride * width
        host[s:s + N * width] = xs[b]
    buf = mq.to_device(host)
    view = buf[off_words:off_words + batch * stride * width]
    return buf, view


@pytest.mark.parametrize("width,bits,log2n,batch,stride_pad,off_words", [
    (3, 188, 14, 4, 0, 1),    # 192-bit residues at an address that is 8- but not 24-byte aligned
    (4, 252, 14, 3, 0, 4),    # 256-bit residues at a 32-byte offset
    (2, 124, 14, 4, 64, 0),   # stride N + 64: staging uses N, the output goes back to the caller's stride
    (1, 60, 15, 3, 3, 1),     # 64-bit residues, odd stride, 8-byte offset
])
def test_noalloc_layouts_match_ntt_forward(mq, width, bits, log2n, batch, stride_pad, off_words):
    """Offsets and strides the staging must respect: the results equal ntt_forward's on the same
    layout, bit for bit, and the words between polynomials stay untouched."""
    import torch
    q = W.gen_prime(bits, log2n + 1, 9)
    psi = W.gen_root(q, log2n, 9)
    N = 1 << log2n
    stride = N + stride_pad
    plan = mq.ntt_plan_create(log2n, q, psi, width, 0)
    for call in range(2):
        x = W.gen_residues(batch * N, q, seed=300 + call, width=width)
        buf_a, view_a = _laid_out(mq, x, batch, N, stride, width, off_words)
        buf_b, view_b = _laid_out(mq, x, batch, N, stride, width, off_words)
        mq.ntt_forward(plan, view_a, batch, stride)
        mq.ntt_forward_noalloc(plan, view_b, batch, stride)
        torch.cuda.synchronize()
        want, got = mq.to_host(buf_a), mq.to_host(buf_b)
        assert np.array_equal(got, want), f"call {call}"
        before, _ = _laid_out(mq, x, batch, N, stride, width, off_words)
        marker = mq.to_host(before) == np.uint64(0x5A5A5A5A5A5A5A5A)
        assert np.array_equal(got[marker], mq.to_host(before)[marker]), "padding between polynomials changed"

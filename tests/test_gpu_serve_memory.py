"""The server's device-memory admission and request cancellation.

Staging (natural-order transforms above 2^12) is the memory the server allocates itself.  A failed
staging allocation -- injected on the host, never provoked on the device -- defers the requests,
which then complete bit-exact; with nothing in flight the staged requests fail with MQ_ERR_OOM after
the wait limit and the server keeps serving; admission follows the free memory the device reports;
a queued request can be cancelled and its buffers stay untouched."""
import time

import numpy as np
import pytest

from paper_2509_12494_gb300 import workload as W

pytestmark = pytest.mark.gpu

LOG2N, N, BATCH = 16, 1 << 16, 4
STAGING = BATCH * N * 16   # bytes of staging one natural-order 124-bit request of BATCH x 2^16 needs
MODES = ["batched", "plain"]


def _sync():
    import torch
    torch.cuda.synchronize()


@pytest.fixture(scope="module")
def case(mq):
    """A natural-order (staged) and a bit-reversed (unstaged) 124-bit plan, one input and its
    forward transform by the per-call path."""
    q = W.gen_prime(124, 18, 31)
    psi = W.gen_root(q, LOG2N, 31)
    nat = mq.ntt_plan_create(LOG2N, q, psi, 2, 0)
    rev = mq.ntt_plan_create(LOG2N, q, psi, 2, mq.MQ_ORDER_BITREV)
    x = W.gen_residues(BATCH * N, q, 31, 2)
    want = {}
    for name, plan in (("nat", nat), ("rev", rev)):
        d = mq.to_device(x)
        mq.ntt_forward(plan, d, BATCH, N)
        _sync()
        want[name] = mq.to_host(d)
    return {"nat": nat, "rev": rev, "x": x, "want": want}


def _cfg(mq, mode, **kw):
    return mq.mq_server_cfg(mode=mq.MQ_SERVE_PLAIN if mode == "plain" else mq.MQ_SERVE_BATCHED, **kw)


def _req(mq, case, order="nat"):
    d = mq.to_device(case["x"])
    return d, mq.ntt_job(mq.MQ_JOB_NTT_FORWARD, case[order], d, BATCH, N)


@pytest.mark.parametrize("mode", MODES)
def test_injected_staging_failures_defer_and_complete(mq, case, mode):
    """Five staging allocations fail; the requests concerned go back to the queue and every request
    still completes, bit-exact, with none failed."""
    srv = mq.mq_server_create(_cfg(mq, mode))
    mq.mq_server_inject_alloc_failures(srv, 5)
    reqs = [_req(mq, case) for _ in range(16)]
    _sync()
    tickets = [mq.mq_submit(srv, j) for _, j in reqs]
    mq.mq_server_drain(srv, 120)
    for (d, _), t in zip(reqs, tickets):
        assert mq.mq_poll(srv, t) == (True, 0)
        assert np.array_equal(mq.to_host(d), case["want"]["nat"])
    st = mq.mq_server_stats(srv)
    assert st["completed"] == 16 and st["failed"] == 0
    assert st["deferred"] >= 5
    if mode == "plain":
        assert st["deferred"] == 5    # one request per failed allocation
    mq.mq_server_destroy(srv)


@pytest.mark.parametrize("mode", MODES)
def test_no_memory_with_nothing_in_flight_fails_after_the_wait_limit(mq, case, mode):
    """Every staging allocation fails: after the wait limit the ten staged requests fail with
    MQ_ERR_OOM -- together, not one wait limit each -- leaving their buffers untouched; requests
    needing no staging, before and behind them, complete; once the failures stop the server serves
    staged requests again."""
    srv = mq.mq_server_create(_cfg(mq, mode, wait_timeout_s=0.2))
    mq.mq_server_inject_alloc_failures(srv, 1 << 30)
    staged = [_req(mq, case) for _ in range(10)]
    d0, j0 = _req(mq, case, "rev")
    d2, j2 = _req(mq, case, "rev")
    _sync()
    t0 = time.perf_counter()
    tr0 = mq.mq_submit(srv, j0)
    ts = [mq.mq_submit(srv, j) for _, j in staged]
    t2 = mq.mq_submit(srv, j2)
    assert all(mq.mq_wait(srv, t, 30) == mq.MQ_ERR_OOM for t in ts)
    elapsed = time.perf_counter() - t0
    assert 0.2 <= elapsed < 1.0, elapsed      # one wait limit, not ten
    assert mq.mq_wait(srv, t2, 30) == 0 and mq.mq_wait(srv, tr0, 30) == 0
    for d, _ in staged:
        assert np.array_equal(mq.to_host(d), case["x"])
    assert np.array_equal(mq.to_host(d0), case["want"]["rev"])
    assert np.array_equal(mq.to_host(d2), case["want"]["rev"])
    mq.mq_server_inject_alloc_failures(srv, 0)
    d3, j3 = _req(mq, case)
    assert mq.mq_wait(srv, mq.mq_submit(srv, j3), 30) == 0
    assert np.array_equal(mq.to_host(d3), case["want"]["nat"])
    st = mq.mq_server_stats(srv)
    assert st["failed"] == 10 and st["completed"] == 3
    mq.mq_server_destroy(srv)


@pytest.mark.parametrize("mode", MODES)
def test_staging_admission_follows_free_device_memory(mq, case, mode):
    """With the reserve at the device's whole memory no staging fits (free memory plus the pool's
    idle bytes never exceed it): the staged request fails with MQ_ERR_OOM after the wait limit,
    while one needing no staging is served.  With the reserve at the free memory less the staging
    and a margin (for allocations between the reading and the server's own), the same request is
    admitted."""
    import torch
    free, total = torch.cuda.mem_get_info()
    srv = mq.mq_server_create(_cfg(mq, mode, wait_timeout_s=0.2, reserve_bytes=total))
    d, j = _req(mq, case)
    _sync()
    assert mq.mq_wait(srv, mq.mq_submit(srv, j), 30) == mq.MQ_ERR_OOM
    assert np.array_equal(mq.to_host(d), case["x"])
    d2, j2 = _req(mq, case, "rev")
    _sync()
    assert mq.mq_wait(srv, mq.mq_submit(srv, j2), 30) == 0
    assert np.array_equal(mq.to_host(d2), case["want"]["rev"])
    mq.mq_server_destroy(srv)

    d, j = _req(mq, case)
    _sync()
    free, total = torch.cuda.mem_get_info()
    srv = mq.mq_server_create(_cfg(mq, mode, wait_timeout_s=0.2,
                                   reserve_bytes=max(1, free - STAGING - (256 << 20))))
    assert mq.mq_wait(srv, mq.mq_submit(srv, j), 30) == 0
    assert np.array_equal(mq.to_host(d), case["want"]["nat"])
    assert mq.mq_server_stats(srv)["failed"] == 0
    mq.mq_server_destroy(srv)


@pytest.mark.parametrize("mode", MODES)
def test_cancel_queued_requests(mq, case, mode):
    """With a budget of one request, requests run one at a time and most of 64 submitted at once
    queue; cancelling the last sixteen finishes each still queued with MQ_ERR_CANCELLED and its
    buffer untouched, while one already launched runs to completion (MQ_ERR_STATE from mq_cancel)."""
    per_request = 2 * STAGING          # operand bytes plus staging
    srv = mq.mq_server_create(_cfg(mq, mode, hbm_budget_bytes=per_request))
    reqs = [_req(mq, case) for _ in range(64)]
    _sync()
    tickets = [mq.mq_submit(srv, j) for _, j in reqs]
    cancelled = set()
    for t in reversed(tickets[-16:]):
        try:
            mq.mq_cancel(srv, t)
            cancelled.add(t)
        except mq.MqError as e:
            assert e.code == mq.MQ_ERR_STATE
    assert cancelled, "nothing was still queued"
    mq.mq_server_drain(srv, 120)
    for (d, _), t in zip(reqs, tickets):
        if t in cancelled:
            assert mq.mq_wait(srv, t, 1) == mq.MQ_ERR_CANCELLED
            assert np.array_equal(mq.to_host(d), case["x"])
        else:
            assert mq.mq_wait(srv, t, 1) == 0
            assert np.array_equal(mq.to_host(d), case["want"]["nat"])
    st = mq.mq_server_stats(srv)
    assert st["cancelled"] == len(cancelled)
    assert st["completed"] == 64 - len(cancelled) and st["failed"] == 0
    assert st["peak_inflight_bytes"] <= per_request
    # a finished ticket, a cancelled one and an unknown one cannot be cancelled
    for t, code in ((tickets[0], mq.MQ_ERR_STATE), (next(iter(cancelled)), mq.MQ_ERR_STATE),
                    (len(tickets) + 5, mq.MQ_ERR_ARG)):
        with pytest.raises(mq.MqError) as e:
            mq.mq_cancel(srv, t)
        assert e.value.code == code
    mq.mq_server_destroy(srv)

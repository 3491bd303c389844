"""The continuous-batching server: every request's result equals the per-call path's (and so the
oracle's, which the per-call tests pin), alone or in a concurrent mix; admission respects the
memory budget; the plain mode gives the same results; bad requests are refused."""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_2509_12494_gb300 import workload as W

pytestmark = pytest.mark.gpu


def _sync():
    import torch
    torch.cuda.synchronize()


class Req:
    """A request with its inputs on the device and its expected result from the per-call path."""

    def __init__(self, M, rng, seed, plans):
        import torch
        self.M = M
        kind = int(rng.integers(0, 6))
        if kind in (0, 1, 5):  # transforms (forward twice as likely), or one of the BLAS ops
            log2n, width, flags = plans[int(rng.integers(0, len(plans)))]
            self.plan, self.q = plans[(log2n, width, flags)]
            self.kind = M.MQ_JOB_NTT_INVERSE if kind == 1 else M.MQ_JOB_NTT_FORWARD
            self.batch = int(rng.integers(1, 3))
            self.N = 1 << log2n
            self.x = W.gen_residues(self.batch * self.N, self.q, seed, width)
            self.d = M.to_device(self.x)
            ref = M.to_device(self.x)
            (M.ntt_inverse if self.kind == 2 else M.ntt_forward)(self.plan, ref, self.batch, self.N)
            _sync()
            self.want = M.to_host(ref)
        else:
            op = ["vadd", "vsub", "vmul", "axpy"][int(rng.integers(0, 4))]
            self.op = op
            width = int(rng.choice([1, 2]))
            self.q = W.gen_prime(60 if width == 1 else 124, 18, seed % 7)
            n = int(rng.integers(1, 1 << 17)) if rng.integers(0, 4) else int(rng.integers(1 << 17, 1 << 21))
            self.a = M.to_device(W.gen_residues(n, self.q, seed * 3 + 1, width))
            b = W.gen_residues(n, self.q, seed * 3 + 2, width)
            self.b = M.to_device(b)
            self.s = W.to_ints(W.gen_residues(1, self.q, seed, width))[0]
            self.kind = {"vadd": 3, "vsub": 4, "vmul": 5, "axpy": 6}[op]
            self.d = self.b if op == "axpy" else torch.empty_like(self.a)
            ref = M.to_device(b) if op == "axpy" else torch.empty_like(self.a)
            if op == "axpy":
                M.mod_axpy(ref, self.s, self.a, n, self.q, width)
            else:
                getattr(M, "mod_" + op)(ref, self.a, self.b, n, self.q, width)
            _sync()
            self.want = M.to_host(ref)
            self.n, self.width = n, width

    def job(self):
        M = self.M
        if self.kind in (1, 2):
            return M.ntt_job(self.kind, self.plan, self.d, self.batch, self.N)
        return M.blas_job(self.kind, self.d, self.a, self.b, self.n, self.q, self.width, self.s)


@pytest.fixture(scope="module")
def plans(mq):
    out = {}
    keys = []
    for log2n in (12, 13, 16, 17):
        for width in (1, 2):
            for flags in (0, 2):
                q = W.gen_prime(60 if width == 1 else 124, 18, log2n + width)
                psi = W.gen_root(q, log2n, 1)
                out[(log2n, width, flags)] = (mq.ntt_plan_create(log2n, q, psi, width, flags), q)
                keys.append((log2n, width, flags))
    out.update({i: k for i, k in enumerate(keys)})
    return _Plans(out, keys)


class _Plans(dict):
    def __init__(self, d, keys):
        super().__init__(d)
        self.keys_ = keys

    def __len__(self):
        return len(self.keys_)

    def __getitem__(self, k):
        if isinstance(k, int):
            return self.keys_[k]
        return dict.__getitem__(self, k)


@pytest.mark.parametrize("mode", ["batched", "plain"])
def test_concurrent_mix_matches_per_call(mq, plans, mode):
    rng = np.random.default_rng(7 if mode == "batched" else 8)
    reqs = [Req(mq, rng, 1000 + i, plans) for i in range(60)]
    cfg = mq.mq_server_cfg(mode=mq.MQ_SERVE_PLAIN if mode == "plain" else mq.MQ_SERVE_BATCHED)
    srv = mq.mq_server_create(cfg)
    tickets = [None] * len(reqs)

    def submit(lo, hi):
        for i in range(lo, hi):
            tickets[i] = mq.mq_submit(srv, reqs[i].job())
            time.sleep(0.0002)

    th = [threading.Thread(target=submit, args=(k, min(k + 20, len(reqs)))) for k in range(0, len(reqs), 20)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    mq.mq_server_drain(srv, 120)
    for r, t in zip(reqs, tickets):
        done, st = mq.mq_poll(srv, t)
        assert done and st == 0
        assert np.array_equal(mq.to_host(r.d), r.want), (r.kind,)
    stats = mq.mq_server_stats(srv)
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    assert 0 < stats["p50_ms"] <= stats["p99_ms"] <= stats["max_ms"]
    if mode == "batched":
        assert stats["batches"] < len(reqs)  # requests were batched together
    mq.mq_server_destroy(srv)


def test_same_result_alone_and_in_the_mix(mq, plans):
    """A request run alone and the same request submitted in the middle of a busy mix give
    bit-identical results."""
    rng = np.random.default_rng(11)
    srv = mq.mq_server_create()
    probe = Req(mq, np.random.default_rng(99), 4242, plans)
    x0 = mq.to_host(probe.d)
    t = mq.mq_submit(srv, probe.job())
    assert mq.mq_wait(srv, t, 60) == 0
    alone = mq.to_host(probe.d)
    assert np.array_equal(alone, probe.want)
    # restore the input and resubmit in the middle of a mix
    probe.d.copy_(mq.to_device(x0).view_as(probe.d))
    _sync()
    mix = [Req(mq, rng, 2000 + i, plans) for i in range(40)]
    tickets = [mq.mq_submit(srv, r.job()) for r in mix[:20]]
    tp = mq.mq_submit(srv, probe.job())
    tickets += [mq.mq_submit(srv, r.job()) for r in mix[20:]]
    mq.mq_server_drain(srv, 120)
    assert mq.mq_poll(srv, tp) == (True, 0)
    assert np.array_equal(mq.to_host(probe.d), alone)
    for r in mix:
        assert np.array_equal(mq.to_host(r.d), r.want)
    mq.mq_server_destroy(srv)


def test_admission_respects_memory_budget(mq, plans):
    """With a budget of a few requests' bytes, requests wait for memory; all still complete."""
    rng = np.random.default_rng(13)
    reqs = [Req(mq, rng, 3000 + i, plans) for i in range(30)]
    budget = 24 << 20
    srv = mq.mq_server_create(mq.mq_server_cfg(hbm_budget_bytes=budget))
    tickets = []
    for r in reqs:
        try:
            tickets.append(mq.mq_submit(srv, r.job()))
        except mq.MqError as e:   # a single request larger than the whole budget is refused
            assert e.code == mq.MQ_ERR_SIZE
            tickets.append(None)
    mq.mq_server_drain(srv, 120)
    stats = mq.mq_server_stats(srv)
    assert stats["peak_inflight_bytes"] <= budget
    for r, t in zip(reqs, tickets):
        if t is not None:
            assert np.array_equal(mq.to_host(r.d), r.want)
    assert sum(t is not None for t in tickets) >= 10
    mq.mq_server_destroy(srv)


def test_server_oracle_spot_check(mq):
    """A served transform against the oracle directly (not only against the per-call path)."""
    q = W.gen_prime(124, 18, 77)
    psi = W.gen_root(q, 12, 77)
    plan = mq.ntt_plan_create(12, q, psi, 2, 0)
    x = W.gen_residues(4096, q, 5, 2)
    d = mq.to_device(x)
    srv = mq.mq_server_create()
    t = mq.mq_submit(srv, mq.ntt_job(1, plan, d, 1, 4096))
    assert mq.mq_wait(srv, t, 60) == 0
    assert np.array_equal(mq.to_host(d), oracle.ntt(x, 12, q, psi, 2))
    mq.mq_server_destroy(srv)


def test_refuses_bad_requests(mq, plans):
    srv = mq.mq_server_create(mq.mq_server_cfg(hbm_budget_bytes=1 << 20))
    plan, q = plans[(16, 2, 0)]
    import torch
    d = torch.zeros((1 << 16, 2), dtype=torch.int64, device="cuda")
    j = mq.ntt_job(1, plan, d, 1, 1 << 16)
    with pytest.raises(mq.MqError) as e:     # 1 MiB + staging > budget of 1 MiB
        mq.mq_submit(srv, j)
    assert e.value.code == mq.MQ_ERR_SIZE
    j.after = 0
    with pytest.raises(mq.MqError) as e:
        mq.mq_submit(srv, j)
    assert e.value.code == mq.MQ_ERR_ARG
    mq.mq_server_destroy(srv)

"""The batched persistent form: every job's result equals the oracle's and the per-call path's,
alone or in a mix, across graph replays and job-table updates; dependency chains; bounded waits."""
import os

import numpy as np
import pytest

import oracle
from paper_2509_12494_gb300 import workload as W
from tests.gpu_util import sample_idx

pytestmark = pytest.mark.gpu


def _sync():
    import torch
    torch.cuda.synchronize()


def _brv(i, bits):
    return int(format(i, f"0{bits}b")[::-1], 2)


class NttCase:
    """A transform job with its inputs, plan and expected output (oracle for small N, sampled
    points from the definition for large N)."""

    def __init__(self, M, log2n, bits, batch, flags, inverse, seed, dseed=None, plan=None):
        self.M, self.log2n, self.batch, self.flags, self.inverse = M, log2n, batch, flags, inverse
        self.width = 2 if bits > 60 else 1
        self.q = W.gen_prime(bits, 18, seed)
        self.psi = W.gen_root(self.q, log2n, seed)
        self.N = 1 << log2n
        self.plan = plan or M.ntt_plan_create(log2n, self.q, self.psi, self.width, flags)
        dseed = seed * 7 + 1 if dseed is None else dseed
        self.x = W.gen_residues(batch * self.N, self.q, seed=dseed, width=self.width)
        self.d = M.to_device(self.x)

    def job(self, after=-1):
        kind = self.M.MQ_JOB_NTT_INVERSE if self.inverse else self.M.MQ_JOB_NTT_FORWARD
        return self.M.ntt_job(kind, self.plan, self.d, self.batch, self.N, after)

    def per_call(self):
        d = self.M.to_device(self.x)
        (self.M.ntt_inverse if self.inverse else self.M.ntt_forward)(self.plan, d, self.batch, self.N)
        _sync()
        return self.M.to_host(d)

    def check_oracle(self, got, pool):
        shp = (self.batch, self.N) if self.width == 1 else (self.batch, self.N, 2)
        g, x = got.reshape(shp), self.x.reshape(shp)
        ofl = (oracle.BITREV if self.flags & 2 else 0)
        if self.log2n <= 12:
            futs = [pool.submit(oracle.ntt, x[b].copy(), self.log2n, self.q, self.psi, self.width, ofl, self.inverse)
                    for b in range(min(self.batch, 2))]
            for b, f in enumerate(futs):
                assert np.array_equal(g[b], f.result()), (self.log2n, b)
        else:
            futs = []
            for b in (0, self.batch - 1):
                for i in sample_idx(self.N, 2, seed=b):
                    i = int(i)
                    if not self.inverse:
                        k = _brv(i, self.log2n) if self.flags & 2 else i
                        futs.append((b, i, pool.submit(oracle.ntt_point, x[b], self.log2n, self.q, self.psi,
                                                       self.width, k)))
                    else:
                        y = x[b] if not self.flags & 2 else x[b][[_brv(k, self.log2n) for k in range(self.N)]]
                        futs.append((b, i, pool.submit(oracle.intt_point, np.ascontiguousarray(y), self.log2n, self.q,
                                                       self.psi, self.width, i)))
            for b, i, f in futs:
                assert W.to_ints(g[b][i:i + 1])[0] == f.result(), (self.log2n, b, i)


class BlasCase:
    KINDS = {"vadd": 3, "vsub": 4, "vmul": 5, "axpy": 6}
    OOPS = {"vadd": oracle.VADD, "vsub": oracle.VSUB, "vmul": oracle.VMUL, "axpy": oracle.AXPY}

    def __init__(self, M, op, n, bits, seed):
        import torch
        self.M, self.op, self.n = M, op, n
        self.width = 2 if bits > 60 else 1
        self.q = W.gen_prime(bits, 18, seed + 50)
        self.a = W.gen_residues(n, self.q, seed=seed * 3 + 1, width=self.width)
        self.b = W.gen_residues(n, self.q, seed=seed * 3 + 2, width=self.width)
        self.s = W.to_ints(W.gen_residues(1, self.q, seed=seed, width=self.width))[0]
        self.da, self.db = M.to_device(self.a), M.to_device(self.b)
        self.dc = self.db if op == "axpy" else torch.empty_like(self.da)

    def job(self, after=-1):
        return self.M.blas_job(self.KINDS[self.op], self.dc, self.da, self.db, self.n, self.q, self.width, self.s, after)

    def expect(self):
        return oracle.blas(self.OOPS[self.op], self.a, self.b, self.q, self.width, s=self.s)


FORMS = ["split", "prefetch", "calls"]
PERSISTENT = ["split", "prefetch"]


def _opts(M, form, **kw):
    """Batch options selecting a form (all must give identical results)."""
    flags = kw.pop("flags", 0) | {"split": M.MQ_BATCH_FORM_SPLIT, "prefetch": M.MQ_BATCH_FORM_PREFETCH,
                                  "calls": M.MQ_BATCH_FORM_CALLS}[form]
    return M.mq_batch_opts(flags=flags, **kw)


def _run(M, jobs, opts=None):
    b = M.mq_batch_create(jobs, opts)
    M.mq_batch_launch(b)
    assert M.mq_batch_status(b) == 0, M.mq_last_error()
    return b


@pytest.mark.parametrize("log2n,bits,flags", [(6, 124, 0), (10, 124, 2), (11, 60, 0), (12, 124, 0), (13, 60, 2),
                                              (16, 124, 2), (16, 124, 0), (17, 60, 0), (17, 124, 2)])
@pytest.mark.parametrize("form", FORMS)
def test_single_job_equals_per_call_and_oracle(mq, pool, log2n, bits, flags, form):
    for inverse in (False, True):
        c = NttCase(mq, log2n, bits, batch=3, flags=flags, inverse=inverse, seed=log2n + bits)
        want = c.per_call()
        _run(mq, [c.job()], _opts(mq, form))
        got = mq.to_host(c.d)
        assert np.array_equal(got, want)
        c.check_oracle(got, pool)


@pytest.mark.parametrize("bits", [124, 60])
@pytest.mark.parametrize("form", FORMS)
def test_uniform_batch_forward_then_inverse(mq, bits, form):
    """Independent transforms, each forward job followed by its inverse in the same launch: the
    forward outputs (checked on a copy) equal the per-call path, the round trip restores x."""
    import torch
    cases = [NttCase(mq, 16, bits, 1, 2, False, 900 + i) for i in range(12)]
    # forward only, to compare spectra
    _run(mq, [c.job() for c in cases], _opts(mq, form))
    for c in cases:
        assert np.array_equal(mq.to_host(c.d), c.per_call())
    # forward then inverse (job 12 + i waits for job i)
    for c in cases:
        c.d.copy_(mq.to_device(c.x))
    jobs = [c.job() for c in cases] + [mq.ntt_job(mq.MQ_JOB_NTT_INVERSE, c.plan, c.d, 1, c.N, after=i)
                                      for i, c in enumerate(cases)]
    b = _run(mq, jobs, _opts(mq, form))
    assert mq.mq_batch_info(b)["ntt_items"] == 24 * 64
    for c in cases:
        assert np.array_equal(mq.to_host(c.d), c.x)
    torch.cuda.synchronize()


@pytest.mark.parametrize("form", FORMS)
def test_uneven_mix_of_sizes_widths_orders_and_blas(mq, pool, form):
    """Transforms of 2^6 .. 2^17, both widths and orders, interleaved with all four BLAS ops of
    ragged lengths: every job's result equals its oracle and per-call result."""
    rng = np.random.default_rng(5)
    ntt, blas = [], []
    for i in range(14):
        log2n = int(rng.integers(6, 18))
        ntt.append(NttCase(mq, log2n, int(rng.choice([60, 124])), int(rng.integers(1, 4)), int(rng.choice([0, 2])),
                           bool(rng.integers(0, 2)), 300 + i))
    for i, op in enumerate(["vadd", "vsub", "vmul", "axpy"] * 3):
        n = int(rng.integers(1, 70000)) if i % 3 else int(rng.integers(16384, 200000))
        blas.append(BlasCase(mq, op, n, int(rng.choice([60, 124])), 400 + i))
    wants = [c.per_call() for c in ntt]
    jobs = []
    for i in range(max(len(ntt), len(blas))):
        if i < len(ntt):
            jobs.append(ntt[i].job())
        if i < len(blas):
            jobs.append(blas[i].job())
    b = _run(mq, jobs, _opts(mq, form, blas_chunk=4096))
    info = mq.mq_batch_info(b)
    assert info["ntt_items"] > 0 and info["blas_items"] > 0
    for c, want in zip(ntt, wants):
        got = mq.to_host(c.d)
        assert np.array_equal(got, want), (c.log2n, c.width, c.flags, c.inverse)
        c.check_oracle(got, pool)
    for c in blas:
        assert np.array_equal(mq.to_host(c.dc), c.expect()), (c.op, c.n, c.width)


@pytest.mark.parametrize("log2n,bits", [(10, 124), (12, 60), (13, 124)])
@pytest.mark.parametrize("form", FORMS)
def test_polynomial_product_chain(mq, log2n, bits, form):
    """forward(a), forward(b) -> vmul -> inverse, as one batch with dependencies, equals the
    schoolbook negacyclic product (Sec. 2.3) computed by the oracle."""
    import torch
    width = 2 if bits > 60 else 1
    q = W.gen_prime(bits, 18, log2n)
    psi = W.gen_root(q, log2n, 1)
    N = 1 << log2n
    plan = mq.ntt_plan_create(log2n, q, psi, width, 2)
    a = W.gen_residues(N, q, 1, width)
    b = W.gen_residues(N, q, 2, width)
    da, db = mq.to_device(a), mq.to_device(b)
    dc = torch.empty_like(da)
    # one `after` per job: fwd(b) waits for fwd(a), so the product that waits for fwd(b) sees both
    jobs = [mq.ntt_job(1, plan, da), mq.ntt_job(1, plan, db, after=0),
            mq.blas_job(mq.MQ_JOB_VMUL, dc, da, db, N, q, width, after=1),
            mq.ntt_job(2, plan, dc, after=2)]
    _run(mq, jobs, _opts(mq, form))
    want = oracle.negacyclic_mul(a, b, log2n, q, width) if log2n <= 12 else None
    got = mq.to_host(dc)
    if want is not None:
        assert np.array_equal(got, want)
    else:  # large N: two sampled coefficients of the schoolbook product
        ai, bi = W.to_ints(a), W.to_ints(b)
        for k in (0, N - 1):
            ref = (sum(ai[i] * bi[k - i] for i in range(k + 1)) - sum(ai[i] * bi[k + N - i] for i in range(k + 1, N))) % q
            assert W.to_ints(got[k:k + 1])[0] == ref


def test_graph_replay_and_update(mq):
    """Replaying the captured graph reruns the jobs; mq_batch_update points them at new buffers."""
    c1 = NttCase(mq, 14, 124, 2, 0, False, 11)
    bl = BlasCase(mq, "vmul", 50001, 124, 12)
    b = mq.mq_batch_create([c1.job(), bl.job()])
    want1 = c1.per_call()
    mq.mq_batch_launch(b)
    assert mq.mq_batch_status(b) == 0
    assert np.array_equal(mq.to_host(c1.d), want1)
    assert np.array_equal(mq.to_host(bl.dc), bl.expect())
    # replay on restored inputs
    c1.d.copy_(mq.to_device(c1.x))
    mq.mq_batch_launch(b)
    assert mq.mq_batch_status(b) == 0
    assert np.array_equal(mq.to_host(c1.d), want1)
    # new buffers, same shapes
    c2 = NttCase(mq, 14, 124, 2, 0, False, 11, dseed=999, plan=c1.plan)  # same plan, new data
    bl2 = BlasCase(mq, "vmul", 50001, 124, 14)
    mq.mq_batch_update(b, [c2.job(), bl2.job()])
    mq.mq_batch_launch(b)
    assert mq.mq_batch_status(b) == 0
    assert np.array_equal(mq.to_host(c2.d), c2.per_call())
    assert np.array_equal(mq.to_host(bl2.dc), bl2.expect())
    # a different shape is refused
    with pytest.raises(mq.MqError):
        mq.mq_batch_update(b, [c2.job()])


def test_no_graph_mode_matches(mq):
    c = NttCase(mq, 15, 60, 2, 2, True, 21)
    want = c.per_call()
    _run(mq, [c.job()], mq.mq_batch_opts(flags=mq.MQ_BATCH_NO_GRAPH))
    assert np.array_equal(mq.to_host(c.d), want)


@pytest.mark.parametrize("form", PERSISTENT)
def test_bounded_wait_reports_timeout_and_device_stays_usable(mq, form):
    """Fault injection: one first-pass item is left out, so the second pass of that polynomial
    waits for a counter nothing will complete.  The wait gives up after the limit, the batch
    reports MQ_ERR_TIMEOUT, and the device keeps working."""
    import time
    c = NttCase(mq, 16, 124, 2, 2, False, 31)
    dep = BlasCase(mq, "vadd", 4096, 124, 32)
    opts = _opts(mq, form, wait_timeout_s=0.2, flags=mq.MQ_BATCH_TEST_DROP_ITEM)
    b = mq.mq_batch_create([c.job(), dep.job(after=0)], opts)
    t0 = time.time()
    mq.mq_batch_launch(b)
    st = mq.mq_batch_status(b)
    assert st == mq.MQ_ERR_TIMEOUT, st
    assert time.time() - t0 < 10
    assert "gave up" in mq.mq_last_error()
    mq.mq_batch_destroy(b)
    # the context is intact: a normal batch still runs and is exact
    c2 = NttCase(mq, 12, 124, 1, 0, False, 33)
    want = c2.per_call()
    _run(mq, [c2.job()])
    assert np.array_equal(mq.to_host(c2.d), want)


@pytest.mark.parametrize("form", PERSISTENT)
def test_instantiation_follows_batch_contents(mq, form):
    """Split form: 64-bit transforms alone run three persistent CTAs per SM, any batch with 128-bit
    residues or BLAS two.  Prefetch form: four for 64-bit transforms alone, three otherwise.  An
    explicit ctas_per_sm is clamped to what the instantiation holds, and the grid to the batch's
    work items.  Each batch's results equal the per-call path's."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    c60 = NttCase(mq, 14, 60, 48, 0, False, 61)    # 768 items: more than any grid holds
    c124 = NttCase(mq, 14, 124, 48, 0, True, 62)
    bl = BlasCase(mq, "vmul", 70001, 60, 63)
    two = 2 if form == "split" else 3
    alone60 = 3 if form == "split" else 4
    for jobs, ctas, kw in (([c60], alone60, {}), ([c124], two, {}), ([c60, c124], two, {}), ([bl], two, {}),
                           ([c60], alone60, {"ctas_per_sm": 7}), ([c124], two, {"ctas_per_sm": 7}),
                           ([c60], 1, {"ctas_per_sm": 1})):
        wants = [j.per_call() if isinstance(j, NttCase) else None for j in jobs]
        for j in jobs:
            if isinstance(j, NttCase):
                j.d.copy_(mq.to_device(j.x).view_as(j.d))
        b = _run(mq, [j.job() for j in jobs], _opts(mq, form, **kw))
        assert mq.mq_batch_info(b)["ctas"] == min(sms * ctas, mq.mq_batch_info(b)["items"])
        for j, w in zip(jobs, wants):
            if w is not None:
                assert np.array_equal(mq.to_host(j.d), w)
            else:
                assert np.array_equal(mq.to_host(j.dc), j.expect())
        mq.mq_batch_destroy(b)


def test_small_batch_takes_the_calls_form(mq):
    """A forward and inverse of one N = 1024 polynomial (two work items): by default the graph holds
    the jobs' own kernels (no persistent grid); equal to the per-call path and to the persistent
    form; a batch with a checked job refuses the calls form and takes a persistent one by default."""
    q = W.gen_prime(124, 11, 5)
    psi = W.gen_root(q, 10, 5)
    plan = mq.ntt_plan_create(10, q, psi, 2, 0)
    x = W.gen_residues(1024, q, 5, width=2)
    d = mq.to_device(x)
    fwd = NttCase(mq, 10, 124, 1, 0, False, 5, plan=plan)
    jobs = [mq.ntt_job(mq.MQ_JOB_NTT_FORWARD, plan, d, 1, 1024), mq.ntt_job(mq.MQ_JOB_NTT_INVERSE, plan, d, 1, 1024, 0)]
    b = _run(mq, jobs)
    assert mq.mq_batch_info(b)["ctas"] == 0
    assert np.array_equal(mq.to_host(d), x)
    # forward alone: equal to the per-call path, in both forms
    for opts in (None, _opts(mq, "prefetch")):
        fwd.d.copy_(mq.to_device(fwd.x))
        bf = _run(mq, [fwd.job()], opts)
        assert (mq.mq_batch_info(bf)["ctas"] == 0) == (opts is None)
        assert np.array_equal(mq.to_host(fwd.d), fwd.per_call())
    checked = mq.ntt_plan_create(10, q, psi, 2, mq.MQ_CHECK_INPUTS)
    cj = [mq.ntt_job(mq.MQ_JOB_NTT_FORWARD, checked, d, 1, 1024)]
    with pytest.raises(mq.MqError) as e:
        mq.mq_batch_create(cj, _opts(mq, "calls"))
    assert e.value.code == mq.MQ_ERR_ARG
    assert mq.mq_batch_info(_run(mq, cj))["ctas"] > 0


def test_rejects_bad_jobs(mq):
    c = NttCase(mq, 10, 124, 1, 0, False, 41)
    with pytest.raises(mq.MqError):
        mq.mq_batch_create([c.job(after=0)])          # depends on itself
    small = NttCase(mq, 4, 124, 1, 0, False, 42)
    with pytest.raises(mq.MqError) as e:
        mq.mq_batch_create([small.job()])              # N below the batched range
    assert e.value.code == mq.MQ_ERR_SIZE


def _restore(cases, bl):
    for c in cases:
        c.d.copy_(c.M.to_device(c.x).view_as(c.d))
    bl.db.copy_(bl.M.to_device(bl.b).view_as(bl.db))


def _check_results(mq, cases, bl):
    for c in cases:
        assert np.array_equal(mq.to_host(c.d), c.per_call()), (c.log2n, c.inverse)
    assert np.array_equal(mq.to_host(bl.dc), bl.expect())


@pytest.mark.parametrize("split_shift", [-1, 0, 1, 3])
@pytest.mark.parametrize("form", FORMS)
def test_every_tuner_axis_is_bit_exact(mq, form, split_shift):
    """Every choice the autotuner can make -- form, stage fusion of two-pass transforms (split_shift,
    clamped to passes of 6..11 stages), CTAs per SM, lag, BLAS chunk -- gives the per-call path's
    results: two-pass transforms of odd and even log N in both orders and directions, with BLAS."""
    cases = [NttCase(mq, 13, 124, 4, 2, False, 70), NttCase(mq, 15, 60, 3, 0, True, 71),
             NttCase(mq, 16, 124, 2, 0, False, 72), NttCase(mq, 17, 60, 1, 2, True, 73)]
    bl = BlasCase(mq, "axpy", 100000, 60, 74)
    jobs = [c.job() for c in cases] + [bl.job()]
    for kw in ({}, {"ctas_per_sm": 1, "lag": 1, "blas_chunk": 8192}):
        _restore(cases, bl)
        b = _run(mq, jobs, _opts(mq, form, split_shift=split_shift, **kw))
        _check_results(mq, cases, bl)
        mq.mq_batch_destroy(b)


def test_autotuner_writes_cache_and_create_uses_it(mq, tmp_path, monkeypatch):
    """The tuner's choice is recorded in the cache under the batch shape; mq_batch_create without
    options takes it from there, and the tuned batch's results equal the per-call path's."""
    import torch
    cases = [NttCase(mq, 13, 124, 4, 2, False, 50 + i) for i in range(2)] + [NttCase(mq, 15, 60, 3, 0, True, 53)]
    bl = BlasCase(mq, "axpy", 100000, 60, 52)
    jobs = [c.job() for c in cases] + [bl.job()]
    cache = str(tmp_path / "tune.json")
    best = mq.mq_autotune_batch(jobs, cache)
    assert best.ctas_per_sm in (1, 2, 3, 4) and best.lag >= 1 and best.blas_chunk % 2048 == 0
    forms = best.flags & (mq.MQ_BATCH_FORM_SPLIT | mq.MQ_BATCH_FORM_PREFETCH | mq.MQ_BATCH_FORM_CALLS)
    assert bin(forms).count("1") == 1 and best.split_shift in (-1, 0, 1)
    text = open(cache).read()
    assert all(k in text for k in ('"ctas_per_sm"', '"form"', '"split"', '"ms"'))
    monkeypatch.setenv("MQNTT_TUNE_CACHE", cache)
    _restore(cases, bl)
    b = _run(mq, jobs)
    info = mq.mq_batch_info(b)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    if forms == mq.MQ_BATCH_FORM_CALLS:
        assert info["ctas"] == 0
    else:
        assert info["ctas"] == min(sms * best.ctas_per_sm, info["items"])
    _check_results(mq, cases, bl)

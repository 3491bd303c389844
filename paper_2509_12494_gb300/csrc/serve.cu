// serve.cu -- the continuous-batching request loop (include/mqntt_serve.h).
//
// One server thread owns the pending queue and `slots` in-flight batches, each with its own
// stream and preallocated device / pinned tables.  Whenever a slot is free it takes the pending
// requests in arrival order while the memory budget allows, expands them into work items
// (build_tables of the batched form), uploads the tables and launches the persistent kernel on the
// slot's stream, followed by a host callback that stamps the completion time.  Natural-order
// transforms above 2^12 get their staging from the library's stream-ordered pool on that stream.
// The plain mode runs each request as its own per-call launch instead, on one stream, with one
// callback per request: the same arrivals through the per-call path, for comparison.
//
// Staging is the memory the server itself allocates, so its admission asks the device: a request
// that needs staging joins a batch only while cudaMemGetInfo's free memory, plus what the pool
// holds unused, less a reserve, covers the batch's staging.  An allocation that fails all the same
// (another process took the memory, or an injected failure) puts the batch's requests back at the
// head of the queue, in order; they wait for requests in flight to free memory, and with nothing
// in flight the first of them that needs staging fails with MQ_ERR_OOM after the wait limit.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/mqntt_serve.h"
#include "batch_internal.h"
#include "plan.h"
#include "trace.h"

int mq_fail(int code, const char *fmt, ...);
int mq_cuda_fail(cudaError_t e, const char *where);
int mq_pool_alloc(void **p, size_t bytes, cudaStream_t s);
int mq_pool_free(void *p, cudaStream_t s);
size_t mq_pool_idle_bytes();

using namespace mq::batch_detail;

static uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

static bool is_ntt_kind(int k) { return k == MQ_JOB_NTT_FORWARD || k == MQ_JOB_NTT_INVERSE; }

namespace {

struct Ticket {
    mq_job job;
    uint64_t t_submit = 0, t_done = 0;
    size_t bytes = 0;
    double butterflies = 0, modmuls = 0;
    int status = MQ_OK;
    bool done = false;
};

struct Server;

struct Slot {
    Server *srv = nullptr;
    cudaStream_t stream = nullptr;
    JobDev *djobs = nullptr, *hjobs = nullptr;
    ItemDev *ditems = nullptr, *hitems = nullptr;
    unsigned *dctrs = nullptr;
    int *h_status = nullptr;
    size_t cap_jobs = 0, cap_items = 0, cap_ctrs = 0;
    std::vector<uint64_t> tickets;
    std::atomic<bool> busy{false}, finished{false};
    std::atomic<uint64_t> t_done{0};
};

struct PlainDone {
    Server *srv;
    uint64_t id;
};

}  // namespace

struct mq_server {
    Server *impl;
};

namespace {

struct Server {
    mq_server_cfg cfg{};
    mq_batch_opts opts{};
    int device = 0;
    unsigned grid = 0;
    size_t smem = 0;
    std::mutex mu;
    std::condition_variable cv;       // wakes the server thread
    std::condition_variable done_cv;  // wakes waiters
    std::deque<uint64_t> pending;
    std::deque<Ticket> tickets;       // ticket id = index + 1
    size_t inflight = 0, peak = 0;
    std::vector<Slot *> slots;
    cudaStream_t plain_stream = nullptr;
    std::atomic<uint64_t> plain_outstanding{0};
    std::thread th;
    bool stop = false;
    std::atomic<unsigned> inject_fail{0};  // staging allocations still to fail (fault injection)
    uint64_t short_since = 0;              // since when staging has been short with nothing in flight
    // statistics since the last reset
    std::vector<double> lat_ms;
    uint64_t completed = 0, failed = 0, batches = 0, batch_jobs = 0, cancelled = 0, deferred = 0;
    uint64_t t_first = 0, t_last = 0;
    double bfly = 0, mm = 0;
    int thread_error = MQ_OK;

    Ticket &ticket(uint64_t id) { return tickets[id - 1]; }

    // Device memory the next staging allocations may take: what the device reports free plus what
    // the library's pool holds unused, less the configured reserve.
    size_t device_available() const {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        const size_t a = fr + mq_pool_idle_bytes();
        return a > cfg.reserve_bytes ? a - cfg.reserve_bytes : 0;
    }

    // A staging allocation on behalf of a request: true when an injected failure is due.
    bool take_injected_failure() {
        unsigned n = inject_fail.load();
        while (n && !inject_fail.compare_exchange_weak(n, n - 1)) {
        }
        return n != 0;
    }

    // Staging could not be had for the queue's first request that needs some.  With requests in
    // flight it waits for them to finish and free theirs; with none, the memory is held outside
    // the server, and once that has lasted the server's wait limit that request fails with
    // MQ_ERR_OOM (and so does each next one short of memory, at once, until a batch launches or
    // the queue empties).  Under mu; true if a request was failed (the caller may try again).
    bool expire_short_head(bool in_flight) {
        auto it = std::find_if(pending.begin(), pending.end(),
                               [&](uint64_t id) { return job_scratch_bytes(ticket(id).job) != 0; });
        if (in_flight || it == pending.end()) {
            short_since = 0;
            return false;
        }
        const uint64_t t = now_ns();
        if (!short_since) short_since = t;
        if ((double)(t - short_since) < cfg.wait_timeout_s * 1e9) return false;
        const uint64_t id = *it;
        pending.erase(it);
        inflight += ticket(id).bytes;  // finish() releases what admission would have held
        finish(id, MQ_ERR_OOM, t);
        return true;
    }

    void finish(uint64_t id, int status, uint64_t t_done) {  // under mu
        Ticket &t = ticket(id);
        t.done = true;
        t.status = status;
        t.t_done = t_done;
        inflight -= t.bytes;
        if (status == MQ_OK) {
            ++completed;
            bfly += t.butterflies;
            mm += t.modmuls;
        } else {
            ++failed;
        }
        lat_ms.push_back((double)(t_done - t.t_submit) * 1e-6);
        if (t_done > t_last) t_last = t_done;
    }
};

void CUDART_CB slot_done_cb(void *arg) {
    Slot *sl = static_cast<Slot *>(arg);
    sl->t_done.store(now_ns());
    sl->finished.store(true);
    {
        std::lock_guard<std::mutex> lk(sl->srv->mu);
    }
    sl->srv->cv.notify_all();
}

void CUDART_CB plain_done_cb(void *arg) {
    PlainDone *p = static_cast<PlainDone *>(arg);
    Server *s = p->srv;
    const uint64_t t = now_ns();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->finish(p->id, MQ_OK, t);
        s->plain_outstanding.fetch_sub(1);
    }
    s->done_cv.notify_all();
    s->cv.notify_all();
    delete p;
}

size_t job_bytes(const mq_job &j) {
    if (is_ntt_kind(j.kind)) {
        size_t op = (j.batch ? j.batch : 1) * ((size_t)1 << j.plan->log2n) * 8u * (size_t)j.plan->width;
        return op + job_scratch_bytes(j);
    }
    return (j.kind == MQ_JOB_AXPY ? 2u : 3u) * j.n * 8u * (size_t)j.width;
}

void job_work(const mq_job &j, double *bfly, double *mm) {
    if (is_ntt_kind(j.kind)) {
        double b = (double)(j.batch ? j.batch : 1) * (double)((size_t)1 << (j.plan->log2n - 1)) * j.plan->log2n;
        *bfly = b;
        *mm = b;
    } else {
        *bfly = 0;
        *mm = (j.kind == MQ_JOB_VMUL || j.kind == MQ_JOB_AXPY) ? (double)j.n : 0.0;
    }
}

int grow(Slot *sl, size_t njobs, size_t nitems, size_t nctrs) {
    cudaError_t e = cudaSuccess;
    if (njobs > sl->cap_jobs) {
        size_t cap = std::max(njobs, 2 * sl->cap_jobs);
        if (sl->djobs) cudaFree(sl->djobs);
        if (sl->hjobs) cudaFreeHost(sl->hjobs);
        sl->djobs = nullptr;
        sl->hjobs = nullptr;
        sl->cap_jobs = 0;
        if ((e = cudaMalloc(&sl->djobs, cap * sizeof(JobDev))) != cudaSuccess ||
            (e = cudaMallocHost(&sl->hjobs, cap * sizeof(JobDev))) != cudaSuccess)
            return mq_fail(MQ_ERR_OOM, "server tables do not fit");
        sl->cap_jobs = cap;
    }
    if (nitems > sl->cap_items) {
        size_t cap = std::max(nitems, 2 * sl->cap_items);
        if (sl->ditems) cudaFree(sl->ditems);
        if (sl->hitems) cudaFreeHost(sl->hitems);
        sl->ditems = nullptr;
        sl->hitems = nullptr;
        sl->cap_items = 0;
        if ((e = cudaMalloc(&sl->ditems, cap * sizeof(ItemDev))) != cudaSuccess ||
            (e = cudaMallocHost(&sl->hitems, cap * sizeof(ItemDev))) != cudaSuccess)
            return mq_fail(MQ_ERR_OOM, "server tables do not fit");
        sl->cap_items = cap;
    }
    if (nctrs > sl->cap_ctrs) {
        size_t cap = std::max(nctrs, 2 * sl->cap_ctrs);
        if (sl->dctrs) cudaFree(sl->dctrs);
        sl->dctrs = nullptr;
        sl->cap_ctrs = 0;
        if ((e = cudaMalloc(&sl->dctrs, cap * sizeof(unsigned))) != cudaSuccess)
            return mq_fail(MQ_ERR_OOM, "server counters do not fit");
        sl->cap_ctrs = cap;
    }
    return MQ_OK;
}

// Build and launch one batch of requests on a free slot (called without the server lock).
int launch_batch(Server *s, Slot *sl, std::vector<mq_job> &jobs) {
    MQ_TRACE("mq_server batch");
    const size_t n = jobs.size();
    std::vector<void *> scratch(n, nullptr);
    int rc = MQ_OK;
    for (size_t i = 0; i < n && !rc; ++i) {
        size_t b = job_scratch_bytes(jobs[i]);
        if (b && s->take_injected_failure())
            rc = mq_fail(MQ_ERR_OOM, "injected staging allocation failure (%zu bytes)", b);
        else if (b)
            rc = mq_pool_alloc(&scratch[i], b, sl->stream);
    }
    BatchTables t;
    unsigned grid = 0;
    size_t smem = 0;
    const int variant = job_variant(jobs.data(), n), form = kernel_form(variant, s->opts.flags);
    if (!rc) rc = persistent_grid(variant, form, 0, &grid, &smem);
    if (!rc) rc = build_tables(jobs.data(), n, s->opts, scratch.data(), 2ull * grid, t);
    if (!rc) rc = grow(sl, n, std::max<size_t>(1, t.items.size()), t.n_ctrs);
    if (!rc) {
        memcpy(sl->hjobs, t.jobs.data(), n * sizeof(JobDev));
        memcpy(sl->hitems, t.items.data(), t.items.size() * sizeof(ItemDev));
        *sl->h_status = 0;
        cudaError_t e;
        if ((e = cudaMemcpyAsync(sl->djobs, sl->hjobs, n * sizeof(JobDev), cudaMemcpyHostToDevice, sl->stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(sl->ditems, sl->hitems, t.items.size() * sizeof(ItemDev), cudaMemcpyHostToDevice,
                                 sl->stream)) != cudaSuccess ||
            (e = launch_persistent(variant, form, sl->djobs, sl->ditems, (unsigned)t.items.size(), sl->dctrs, t.n_ctrs,
                                   (unsigned)n, (unsigned long long)(s->opts.wait_timeout_s * 1e9), grid, smem,
                                   sl->stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(sl->h_status, sl->dctrs + 1, sizeof(int), cudaMemcpyDeviceToHost, sl->stream)) !=
                cudaSuccess)
            rc = mq_cuda_fail(e, "server batch launch");
    }
    for (size_t i = 0; i < n; ++i)
        if (scratch[i]) mq_pool_free(scratch[i], sl->stream);  // stream-ordered after the kernel
    if (!rc) {
        cudaError_t e = cudaLaunchHostFunc(sl->stream, slot_done_cb, sl);
        if (e != cudaSuccess) rc = mq_cuda_fail(e, "server completion callback");
    }
    return rc;
}

int run_plain(Server *s, uint64_t id) {
    MQ_TRACE("mq_server plain request");
    const mq_job &j = s->ticket(id).job;
    void *st = (void *)s->plain_stream;
    if (job_scratch_bytes(j) && s->take_injected_failure())
        return mq_fail(MQ_ERR_OOM, "injected staging allocation failure (%zu bytes)", job_scratch_bytes(j));
    int rc;
    switch (j.kind) {
    case MQ_JOB_NTT_FORWARD: rc = ntt_forward(j.plan, j.data, j.batch ? j.batch : 1, j.stride, st); break;
    case MQ_JOB_NTT_INVERSE: rc = ntt_inverse(j.plan, j.data, j.batch ? j.batch : 1, j.stride, st); break;
    case MQ_JOB_VADD: rc = mod_vadd(j.data, j.a, j.b, j.n, j.q, j.width, st); break;
    case MQ_JOB_VSUB: rc = mod_vsub(j.data, j.a, j.b, j.n, j.q, j.width, st); break;
    case MQ_JOB_VMUL: rc = mod_vmul(j.data, j.a, j.b, j.n, j.q, j.width, st); break;
    default: rc = mod_axpy(j.data, j.scalar, j.a, j.n, j.q, j.width, st); break;
    }
    if (rc) return rc;
    PlainDone *p = new PlainDone{s, id};
    cudaError_t e = cudaLaunchHostFunc(s->plain_stream, plain_done_cb, p);
    if (e != cudaSuccess) {
        delete p;
        return mq_cuda_fail(e, "plain completion callback");
    }
    return MQ_OK;
}

void server_loop(Server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        // completions of batches
        for (Slot *sl : s->slots) {
            if (sl->busy.load() && sl->finished.load()) {
                const int st = *(volatile int *)sl->h_status;
                const uint64_t t = sl->t_done.load();
                for (uint64_t id : sl->tickets) s->finish(id, st, t);
                sl->tickets.clear();
                sl->finished.store(false);
                sl->busy.store(false);
                s->done_cv.notify_all();
            }
        }
        bool any_busy = false;
        for (Slot *sl : s->slots) any_busy |= sl->busy.load();
        if (s->stop && s->pending.empty() && !any_busy && s->plain_outstanding.load() == 0) break;

        // dispatch
        if (s->pending.empty()) s->short_since = 0;
        if (s->cfg.mode == MQ_SERVE_PLAIN) {
            size_t avail = 0;  // staging the device can still give in this pass (asked once per pass)
            bool asked = false;
            while (!s->pending.empty()) {
                const uint64_t id = s->pending.front();
                Ticket &t = s->ticket(id);
                const bool others = s->plain_outstanding.load() > 0;
                if (s->inflight + t.bytes > s->cfg.hbm_budget_bytes && others) break;
                const size_t sb = job_scratch_bytes(t.job);
                if (sb) {
                    if (!asked) {
                        avail = s->device_available();
                        asked = true;
                    }
                    if (sb > avail) {  // the device cannot hold its staging now
                        if (s->expire_short_head(others)) continue;
                        break;
                    }
                    avail -= sb;
                }
                s->pending.pop_front();
                s->inflight += t.bytes;
                s->peak = std::max(s->peak, s->inflight);
                s->plain_outstanding.fetch_add(1);
                ++s->batches;
                ++s->batch_jobs;
                lk.unlock();
                int rc = run_plain(s, id);
                lk.lock();
                if (rc == MQ_ERR_OOM) {  // nothing was launched: back to the head of the queue
                    s->inflight -= t.bytes;
                    s->pending.push_front(id);
                    s->plain_outstanding.fetch_sub(1);
                    --s->batches;
                    --s->batch_jobs;
                    ++s->deferred;
                    s->expire_short_head(s->plain_outstanding.load() > 0);
                    break;
                }
                s->short_since = 0;
                if (rc) {
                    s->finish(id, rc, now_ns());
                    s->plain_outstanding.fetch_sub(1);
                    s->done_cv.notify_all();
                }
            }
        } else {
            for (Slot *sl : s->slots) {
                if (sl->busy.load() || s->pending.empty()) continue;
                if (s->cfg.linger_us > 0 && s->pending.size() < s->cfg.max_batch_jobs) {
                    const uint64_t age = now_ns() - s->ticket(s->pending.front()).t_submit;
                    if ((double)age < s->cfg.linger_us * 1e3 && any_busy) break;
                }
                std::vector<mq_job> jobs;
                size_t staging = 0, avail = 0;
                bool asked = false, short_of_memory = false;
                while (!s->pending.empty() && jobs.size() < s->cfg.max_batch_jobs) {
                    Ticket &t = s->ticket(s->pending.front());
                    if (s->inflight + t.bytes > s->cfg.hbm_budget_bytes) break;  // wait for the budget to free up
                    const size_t sb = job_scratch_bytes(t.job);
                    if (sb) {  // staging comes from device memory: take it only while the device has it
                        if (!asked) {
                            avail = s->device_available();
                            asked = true;
                        }
                        if (staging + sb > avail) {
                            short_of_memory = true;
                            break;
                        }
                        staging += sb;
                    }
                    s->inflight += t.bytes;
                    jobs.push_back(t.job);
                    sl->tickets.push_back(s->pending.front());
                    s->pending.pop_front();
                }
                if (jobs.empty()) {
                    if (short_of_memory && s->expire_short_head(any_busy)) continue;
                    break;
                }
                s->peak = std::max(s->peak, s->inflight);
                sl->busy.store(true);
                ++s->batches;
                s->batch_jobs += jobs.size();
                lk.unlock();
                int rc = launch_batch(s, sl, jobs);
                lk.lock();
                if (rc == MQ_ERR_OOM) {  // nothing was launched: the requests go back to the head of the queue
                    for (auto it = sl->tickets.rbegin(); it != sl->tickets.rend(); ++it) {
                        s->inflight -= s->ticket(*it).bytes;
                        s->pending.push_front(*it);
                    }
                    s->deferred += sl->tickets.size();
                    --s->batches;
                    s->batch_jobs -= jobs.size();
                    sl->tickets.clear();
                    sl->busy.store(false);
                    bool in_flight = false;
                    for (Slot *o : s->slots) in_flight |= o->busy.load();
                    s->expire_short_head(in_flight);
                    break;
                }
                if (!rc) s->short_since = 0;  // a batch launched: the shortage, if any, is over
                if (rc) {
                    const uint64_t t = now_ns();
                    for (uint64_t id : sl->tickets) s->finish(id, rc, t);
                    sl->tickets.clear();
                    sl->busy.store(false);
                    s->done_cv.notify_all();
                }
                any_busy = true;
            }
        }
        s->cv.wait_for(lk, std::chrono::microseconds(100));
    }
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------------

extern "C" int mq_server_create(mq_server **out, const mq_server_cfg *cfg) {
    if (!out) return mq_fail(MQ_ERR_ARG, "out is NULL");
    *out = nullptr;
    Server *s = new Server();
    if (cfg) s->cfg = *cfg;
    if (s->cfg.mode != MQ_SERVE_BATCHED && s->cfg.mode != MQ_SERVE_PLAIN) {
        delete s;
        return mq_fail(MQ_ERR_ARG, "unknown server mode %d", s->cfg.mode);
    }
    cudaError_t ge = cudaGetDevice(&s->device);
    if (ge != cudaSuccess) {
        delete s;
        return mq_cuda_fail(ge, "cudaGetDevice");
    }
    if (s->cfg.hbm_budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        if ((ge = cudaMemGetInfo(&fr, &tot)) != cudaSuccess) {
            delete s;
            return mq_cuda_fail(ge, "cudaMemGetInfo");
        }
        s->cfg.hbm_budget_bytes = fr / 2;
    }
    if (s->cfg.reserve_bytes == 0) s->cfg.reserve_bytes = (size_t)256 << 20;
    if (s->cfg.slots == 0) s->cfg.slots = 2;
    if (s->cfg.max_batch_jobs == 0) s->cfg.max_batch_jobs = 4096;
    if (s->cfg.wait_timeout_s <= 0) s->cfg.wait_timeout_s = 2.0;
    s->opts.wait_timeout_s = s->cfg.wait_timeout_s;
    apply_defaults(s->opts);
    int rc = persistent_grid(3, 0, 0, &s->grid, &s->smem);  // the general instantiation must fit
    if (rc) {
        delete s;
        return rc;
    }
    cudaError_t e = cudaStreamCreateWithFlags(&s->plain_stream, cudaStreamNonBlocking);
    for (unsigned i = 0; i < s->cfg.slots && e == cudaSuccess; ++i) {
        Slot *sl = new Slot();
        sl->srv = s;
        s->slots.push_back(sl);
        if ((e = cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking)) != cudaSuccess) break;
        e = cudaMallocHost(&sl->h_status, sizeof(int));
    }
    if (e != cudaSuccess) {
        mq_server tmp{s};
        mq_server_destroy(new mq_server(tmp));
        return mq_cuda_fail(e, "server streams");
    }
    s->th = std::thread(server_loop, s);
    *out = new mq_server{s};
    return MQ_OK;
}

extern "C" int mq_submit(mq_server *srv, const mq_job *job, uint64_t *ticket) {
    if (!srv || !job || !ticket) return mq_fail(MQ_ERR_ARG, "NULL argument");
    Server *s = srv->impl;
    if (job->after != -1) return mq_fail(MQ_ERR_ARG, "served jobs are independent: `after` must be -1");
    if (is_ntt_kind(job->kind) && !job->plan) return mq_fail(MQ_ERR_ARG, "NTT job without a plan");
    // a failed check would fail every request batched with this one: served jobs are not checked
    if ((is_ntt_kind(job->kind) && (job->plan->flags & MQ_CHECK_INPUTS)) ||
        (!is_ntt_kind(job->kind) && ((unsigned)job->width & MQ_CHECK_INPUTS)))
        return mq_fail(MQ_ERR_ARG, "the server does not take jobs with MQ_CHECK_INPUTS: check inputs before submitting");
    {
        int rc = check_job(*job, s->opts);  // everything a batch would check about this job
        if (rc) return rc;
    }
    Ticket t;
    t.job = *job;
    t.bytes = job_bytes(*job);
    job_work(*job, &t.butterflies, &t.modmuls);
    if (t.bytes > s->cfg.hbm_budget_bytes)
        return mq_fail(MQ_ERR_SIZE, "the job needs %zu bytes, more than the server's whole budget (%zu)", t.bytes,
                       s->cfg.hbm_budget_bytes);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        t.t_submit = now_ns();
        if (s->t_first == 0) s->t_first = t.t_submit;
        s->tickets.push_back(t);
        *ticket = s->tickets.size();
        s->pending.push_back(*ticket);
    }
    s->cv.notify_all();
    return MQ_OK;
}

// splitmix64: a small seeded generator for the arrival process
static uint64_t splitmix64(uint64_t &x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

extern "C" int mq_server_poisson(mq_server *srv, const mq_job *pool, size_t npool, double rate_per_s,
                                 uint64_t n_requests, uint64_t seed, double *offered_per_s) {
    if (!srv || !pool || !npool) return mq_fail(MQ_ERR_ARG, "NULL or empty request pool");
    std::vector<uint64_t> last(npool, 0);
    uint64_t st = seed;
    const uint64_t t0 = now_ns();
    double t_next = 0.0;  // ns after t0
    for (uint64_t i = 0; i < n_requests; ++i) {
        if (rate_per_s > 0) {
            // exponential inter-arrival time by inversion of a uniform draw in (0, 1]
            const double u = ((double)(splitmix64(st) >> 11) + 1.0) * (1.0 / 9007199254740992.0);
            t_next += -std::log(u) / rate_per_s * 1e9;
            while ((double)(now_ns() - t0) < t_next) {
            }
        }
        const size_t k = (size_t)(i % npool);
        if (last[k]) {  // a request's buffers are not reused while it is in flight
            int status = 0;
            int rc = mq_wait(srv, last[k], 600.0, &status);
            if (rc) return rc;
        }
        int rc = mq_submit(srv, &pool[k], &last[k]);
        if (rc) return rc;
    }
    if (offered_per_s) *offered_per_s = (double)n_requests / ((double)(now_ns() - t0) * 1e-9);
    return MQ_OK;
}

extern "C" int mq_cancel(mq_server *srv, uint64_t ticket) {
    if (!srv) return mq_fail(MQ_ERR_ARG, "NULL server");
    Server *s = srv->impl;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (ticket == 0 || ticket > s->tickets.size())
            return mq_fail(MQ_ERR_ARG, "unknown ticket %llu", (unsigned long long)ticket);
        auto it = std::find(s->pending.begin(), s->pending.end(), ticket);
        if (it == s->pending.end())
            return mq_fail(MQ_ERR_STATE, "ticket %llu is no longer queued (launched or finished)",
                           (unsigned long long)ticket);
        s->pending.erase(it);
        Ticket &t = s->ticket(ticket);
        t.done = true;
        t.status = MQ_ERR_CANCELLED;
        t.t_done = now_ns();
        ++s->cancelled;
    }
    s->done_cv.notify_all();
    s->cv.notify_all();
    return MQ_OK;
}

extern "C" int mq_server_inject_alloc_failures(mq_server *srv, unsigned n) {
    if (!srv) return mq_fail(MQ_ERR_ARG, "NULL server");
    srv->impl->inject_fail.store(n);
    srv->impl->cv.notify_all();
    return MQ_OK;
}

extern "C" int mq_poll(mq_server *srv, uint64_t ticket, int *done, int *status) {
    if (!srv || !done) return mq_fail(MQ_ERR_ARG, "NULL argument");
    Server *s = srv->impl;
    std::lock_guard<std::mutex> lk(s->mu);
    if (ticket == 0 || ticket > s->tickets.size()) return mq_fail(MQ_ERR_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    const Ticket &t = s->ticket(ticket);
    *done = t.done;
    if (status) *status = t.done ? t.status : MQ_OK;
    return MQ_OK;
}

extern "C" int mq_wait(mq_server *srv, uint64_t ticket, double timeout_s, int *status) {
    if (!srv) return mq_fail(MQ_ERR_ARG, "NULL server");
    Server *s = srv->impl;
    std::unique_lock<std::mutex> lk(s->mu);
    if (ticket == 0 || ticket > s->tickets.size()) return mq_fail(MQ_ERR_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (!s->ticket(ticket).done) {
        if (s->done_cv.wait_until(lk, deadline) == std::cv_status::timeout && !s->ticket(ticket).done)
            return mq_fail(MQ_ERR_TIMEOUT, "ticket %llu not done after %.3f s", (unsigned long long)ticket, timeout_s);
    }
    if (status) *status = s->ticket(ticket).status;
    return MQ_OK;
}

extern "C" int mq_server_drain(mq_server *srv, double timeout_s) {
    if (!srv) return mq_fail(MQ_ERR_ARG, "NULL server");
    Server *s = srv->impl;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    for (;;) {
        bool all = true;
        for (const Ticket &t : s->tickets) all &= t.done;
        if (all) return MQ_OK;
        if (s->done_cv.wait_until(lk, deadline) == std::cv_status::timeout) {
            bool all2 = true;
            for (const Ticket &t : s->tickets) all2 &= t.done;
            return all2 ? MQ_OK : mq_fail(MQ_ERR_TIMEOUT, "server not drained after %.3f s", timeout_s);
        }
    }
}

extern "C" int mq_server_stats(mq_server *srv, mq_stats *out) {
    if (!srv || !out) return mq_fail(MQ_ERR_ARG, "NULL argument");
    Server *s = srv->impl;
    std::lock_guard<std::mutex> lk(s->mu);
    memset(out, 0, sizeof *out);
    out->submitted = s->tickets.size();
    out->completed = s->completed;
    out->failed = s->failed;
    out->batches = s->batches;
    out->cancelled = s->cancelled;
    out->deferred = s->deferred;
    out->peak_inflight_bytes = s->peak;
    out->mean_batch_jobs = s->batches ? (double)s->batch_jobs / (double)s->batches : 0.0;
    std::vector<double> v = s->lat_ms;
    if (!v.empty()) {
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            size_t k = (size_t)std::min<double>((double)(v.size() - 1), std::max(0.0, p * (double)v.size() - 1.0 + 0.5));
            return v[k];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        out->max_ms = v.back();
        double sum = 0;
        for (double x : v) sum += x;
        out->mean_ms = sum / (double)v.size();
    }
    if (s->t_last > s->t_first) {
        out->span_s = (double)(s->t_last - s->t_first) * 1e-9;
        out->jobs_per_s = (double)s->completed / out->span_s;
        out->butterflies_per_s = s->bfly / out->span_s;
        out->modmul_per_s = s->mm / out->span_s;
    }
    return MQ_OK;
}

extern "C" int mq_server_reset_stats(mq_server *srv) {
    if (!srv) return mq_fail(MQ_ERR_ARG, "NULL server");
    Server *s = srv->impl;
    std::lock_guard<std::mutex> lk(s->mu);
    s->lat_ms.clear();
    s->completed = s->failed = s->batches = s->batch_jobs = s->cancelled = s->deferred = 0;
    s->t_first = s->t_last = 0;
    s->bfly = s->mm = 0;
    s->peak = s->inflight;
    return MQ_OK;
}

extern "C" int mq_server_destroy(mq_server *srv) {
    if (!srv) return MQ_OK;
    Server *s = srv->impl;
    if (s->th.joinable()) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv.notify_all();
        s->th.join();
    }
    cudaDeviceSynchronize();
    for (Slot *sl : s->slots) {
        if (sl->stream) cudaStreamDestroy(sl->stream);
        if (sl->djobs) cudaFree(sl->djobs);
        if (sl->ditems) cudaFree(sl->ditems);
        if (sl->dctrs) cudaFree(sl->dctrs);
        if (sl->hjobs) cudaFreeHost(sl->hjobs);
        if (sl->hitems) cudaFreeHost(sl->hitems);
        if (sl->h_status) cudaFreeHost(sl->h_status);
        delete sl;
    }
    if (s->plain_stream) cudaStreamDestroy(s->plain_stream);
    delete s;
    delete srv;
    return MQ_OK;
}

/*
 * mqntt_serve.h -- a continuous-batching request loop for transforms and BLAS operations.
 *
 * Clients submit single jobs (an NTT of a plan, or one BLAS operation) over device buffers they own
 * and keep resident; plans (twiddle tables) stay resident too.  A server thread admits requests by
 * device memory, twice over: each in-flight request holds its operand bytes, plus staging for
 * natural-order transforms above 2^12, against a budget; and the staging, which the server
 * allocates itself, is taken only while the device has it (cudaMemGetInfo's free memory plus what
 * the library's pool holds unused, less `reserve_bytes`).  A staging allocation that fails all the
 * same defers the batch's requests to the head of the queue, where they wait for requests in flight
 * to free memory; with nothing in flight the first of them that needs staging fails with
 * MQ_ERR_OOM after the wait limit.  The server forms batches of whatever has arrived whenever an
 * in-flight slot is free, launching each batch as one persistent kernel (mqntt_batch.h) on the
 * slot's own stream.  Requests that arrive while other batches run join the next batch, so their
 * work overlaps on the device with the batches already running.  Every result is the same as the
 * per-call entry points give (integer arithmetic; no tolerance).  Latency is measured per request
 * from mq_submit to the completion of its batch, observed by a host callback on the slot's stream.
 *
 * The paper measures single kernels on one CPU core (its Sec. 5) and notes that real FHE workloads
 * batch many independent NTT and BLAS calls (Sec. 6); this loop is the serving form of that
 * batching.
 */
#ifndef MQNTT_SERVE_H
#define MQNTT_SERVE_H

#include "mqntt_batch.h"

#ifdef __cplusplus
extern "C" {
#endif

#define MQ_SERVE_BATCHED 0 /* continuous batching into persistent launches */
#define MQ_SERVE_PLAIN 1   /* one per-call launch per request, in arrival order, on one stream */

typedef struct mq_server_cfg {
    size_t hbm_budget_bytes;  /* in-flight request bytes allowed (0: half the free device memory) */
    unsigned slots;           /* batches in flight at once, each on its own stream (0: 2) */
    unsigned max_batch_jobs;  /* requests per batch (0: 4096) */
    double linger_us;         /* with a slot free, wait up to this long for more arrivals (0: none) */
    double wait_timeout_s;    /* limit of the device-side waits (0: 2 s) */
    int mode;                 /* MQ_SERVE_BATCHED or MQ_SERVE_PLAIN */
    size_t reserve_bytes;     /* device memory staging allocations leave free (0: 256 MiB) */
} mq_server_cfg;

typedef struct mq_stats {
    uint64_t submitted, completed, failed, batches;
    double p50_ms, p99_ms, mean_ms, max_ms; /* latency, submit -> completion */
    double span_s;                          /* first submission to last completion */
    double jobs_per_s;                      /* completed / span */
    double butterflies_per_s;               /* butterflies of completed transforms / span */
    double modmul_per_s;                    /* modular products (butterflies, vmul and axpy elements) / span */
    double mean_batch_jobs;
    size_t peak_inflight_bytes;
    uint64_t cancelled;                     /* requests cancelled while queued (not in the latencies) */
    uint64_t deferred;                      /* requests sent back to the queue by a failed staging allocation */
} mq_stats;

typedef struct mq_server mq_server;

/* Start a server (its thread and streams) on the current device. `cfg` may be NULL (defaults). */
int mq_server_create(mq_server **out, const mq_server_cfg *cfg);

/*
 * Submit one job (mq_job of mqntt_batch.h; `after` must be -1).  Returns at once with a ticket.
 * The job's buffers (and plan) must stay valid and untouched until the ticket completes.  A job
 * larger than the whole budget is rejected with MQ_ERR_SIZE; other argument errors are reported
 * here (MQ_ERR_ARG, MQ_ERR_ALIGN, MQ_ERR_MODULUS, MQ_ERR_RANGE).  A ticket finishes with MQ_OK,
 * MQ_ERR_CANCELLED (mq_cancel), MQ_ERR_OOM (no staging memory with nothing in flight, after the wait
 * limit), MQ_ERR_TIMEOUT (a device-side wait of its batch gave up) or the error of its launch.
 */
int mq_submit(mq_server *s, const mq_job *job, uint64_t *ticket);

/*
 * Cancel a request that is still queued: it finishes at once with status MQ_ERR_CANCELLED, and its
 * buffers are not touched.  MQ_ERR_STATE if it already joined a launched batch or finished (it then
 * runs to completion as usual); MQ_ERR_ARG for an unknown ticket.
 */
int mq_cancel(mq_server *s, uint64_t ticket);

/*
 * Fault injection for tests: the server's next `n` staging allocations report failure as if the
 * device were out of memory (0 clears it).  Nothing on the device is touched; the requests concerned
 * are deferred as a real failure would defer them.
 */
int mq_server_inject_alloc_failures(mq_server *s, unsigned n);

/* Non-blocking: *done = 1 once the ticket finished; *status = its status (MQ_OK or an error). */
int mq_poll(mq_server *s, uint64_t ticket, int *done, int *status);

/* Block until the ticket finishes (or `timeout_s` passes: MQ_ERR_TIMEOUT); *status as mq_poll. */
int mq_wait(mq_server *s, uint64_t ticket, double timeout_s, int *status);

/* Block until every submitted ticket finished (MQ_ERR_TIMEOUT after `timeout_s`). */
int mq_server_drain(mq_server *s, double timeout_s);

/*
 * Open-loop load generator: submit `n_requests` requests taken round-robin from `pool`, with
 * exponential inter-arrival times of mean 1/rate_per_s (a Poisson process drawn from `seed`;
 * rate_per_s <= 0 submits as fast as possible).  A pool entry is resubmitted only after its
 * previous request finished (its buffers are reused).  Returns once all are submitted, with the
 * achieved submission rate in *offered_per_s (may be NULL); use mq_server_drain to wait for them.
 */
int mq_server_poisson(mq_server *s, const mq_job *pool, size_t npool, double rate_per_s, uint64_t n_requests,
                      uint64_t seed, double *offered_per_s);

/* Statistics over the tickets completed since creation or the last reset. */
int mq_server_stats(mq_server *s, mq_stats *out);
int mq_server_reset_stats(mq_server *s);

/* Drain, stop the thread, free everything.  NULL is accepted. */
int mq_server_destroy(mq_server *s);

#ifdef __cplusplus
}
#endif

#endif /* MQNTT_SERVE_H */

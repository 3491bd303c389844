/*
 * mqntt_batch.h -- many transforms and BLAS operations in one persistent, graph-captured launch.
 *
 * Real FHE workloads run many independent NTTs and BLAS operations at once; the paper names
 * batching them as the way to reach the speed of light of a whole processor (Sec. 6, the
 * paragraph on realising the speed of light).  A batch describes up to millions of
 * work items over jobs of uneven sizes, moduli and widths; one persistent kernel pulls the items
 * from a device counter, each job waiting (with a bounded wait) only for what it depends on.  The
 * launch is captured in a CUDA graph once; later launches replay it, and mq_batch_update rewrites
 * the job table (pointers, scalars) without re-capturing.  The arithmetic is the same as the
 * per-call entry points of mqntt.h, so every job's result is bit-identical to running it alone.
 *
 * Requirements: NTT jobs need 2^6 <= N <= 2^22 (use ntt_forward / ntt_inverse otherwise); all
 * device pointers aligned to 16 bytes; BLAS 64-bit residues of length >= 1.
 *
 * Input checking (MQ_CHECK_INPUTS of mqntt.h; Sec. 2.1's canonical operands): NTT jobs whose plan
 * carries the flag and BLAS jobs whose `width` carries it (width = MQ_W128 | MQ_CHECK_INPUTS) have
 * their inputs range-checked by a kernel in the launch, before any job runs.  If a residue is >= q,
 * no job of the batch runs (every output is untouched) and mq_batch_status returns MQ_ERR_RANGE.
 * The check sees the buffers as they are when the launch starts: an input that an earlier job of
 * the same batch writes is checked as it was before the batch.  The server (mqntt_serve.h) does not
 * take checked jobs.
 */
#ifndef MQNTT_BATCH_H
#define MQNTT_BATCH_H

#include "mqntt.h"

#ifdef __cplusplus
extern "C" {
#endif

/* job kinds */
#define MQ_JOB_NTT_FORWARD 1 /* in-place ntt_forward(plan, data, batch, stride) */
#define MQ_JOB_NTT_INVERSE 2 /* in-place ntt_inverse(plan, data, batch, stride) */
#define MQ_JOB_VADD 3        /* data = a + b mod q */
#define MQ_JOB_VSUB 4        /* data = a - b mod q */
#define MQ_JOB_VMUL 5        /* data = a * b mod q */
#define MQ_JOB_AXPY 6        /* data = scalar * a + data mod q (y = data, x = a) */

typedef struct mq_job {
    int kind;             /* MQ_JOB_* */
    int after;            /* index of an earlier job of the same batch that must finish first, or -1 */
    const ntt_plan *plan; /* NTT jobs: plan (modulus, root, size, order) */
    void *data;           /* NTT: polynomials, transformed in place; BLAS: the output vector */
    const void *a;        /* BLAS: first input (axpy: x) */
    const void *b;        /* BLAS: second input (vadd/vsub/vmul) */
    size_t n;             /* BLAS: residues */
    size_t batch;         /* NTT: polynomials */
    size_t stride;        /* NTT: residues between consecutive polynomials (>= N; ignored if batch = 1) */
    uint64_t q[2];        /* BLAS: modulus, low word first */
    uint64_t scalar[2];   /* axpy: the scalar (< q) */
    int width;            /* BLAS: MQ_W64 or MQ_W128 (NTT jobs take the plan's) */
} mq_job;

/* batch creation options; zero-initialised fields take the defaults */
typedef struct mq_batch_opts {
    unsigned ctas_per_sm;  /* persistent CTAs per SM (0: as many as fit -- 3 with the prefetching form,
                              4 for batches of 64-bit transforms only; 2 and 3 with the split form;
                              larger values are clamped to that) */
    unsigned lag;          /* pipeline lag between dependent stages, in waves of the persistent grid (0: 32) */
    unsigned blas_chunk;   /* residues per BLAS work item (0: 16384); a multiple of 2048 */
    double wait_timeout_s; /* limit of every device-side wait (0: 2 s) */
    unsigned flags;        /* MQ_BATCH_* */
    int split_shift;       /* stage fusion of transforms above 2^11: the first pass (columns of the
                              forward, undone last by the inverse) fuses floor(log2 N / 2) + split_shift
                              stages, the second the rest; clamped so that both passes hold 6 to 11
                              stages (0: the even split).  Results do not depend on it. */
} mq_batch_opts;

#define MQ_BATCH_NO_GRAPH 1u       /* launch the kernel directly instead of replaying a graph */
#define MQ_BATCH_TEST_DROP_ITEM 2u /* fault injection for tests: leave out the first first-pass item of the
                                      first two-pass NTT job, so that its dependants' waits run out and
                                      mq_batch_status reports MQ_ERR_TIMEOUT */
/* Kernel form (neither flag: the library's default for the batch's contents).  Both compute the same
   results; they differ in how a CTA overlaps the loads of its next item with the current one. */
#define MQ_BATCH_FORM_SPLIT 4u    /* warp-specialised: two producer warps stage items for eight compute warps */
#define MQ_BATCH_FORM_PREFETCH 8u /* every warp computes; a CTA starts its next item's copies before the
                                     current transform when that item's dependencies are already met */
#define MQ_BATCH_FORM_CALLS 16u   /* no persistent kernel: the graph holds each job's own kernels (the
                                     transform passes and BLAS kernels of the per-call entry points), in job
                                     order.  The default for a batch with fewer work items than the GPU has
                                     SMs and no checked job, where a persistent grid would mostly idle;
                                     refused (MQ_ERR_ARG) for a batch with checked jobs */

typedef struct mq_batch mq_batch;

/*
 * Build a batch over `njobs` jobs: validate them, expand them into work items, upload the job and
 * item tables, allocate the batch's counters and any staging (natural-order NTT jobs above 2^12),
 * and capture the launch in a graph on an internal stream.  `opts` may be NULL (defaults, or the
 * autotuner's cached choice for this batch shape when MQNTT_TUNE_CACHE names a cache file).
 * The batch keeps no reference to `jobs`.  Synchronises `stream`.
 * Errors: MQ_ERR_ARG (bad kind, dependency not earlier, size), MQ_ERR_MODULUS, MQ_ERR_ALIGN,
 * MQ_ERR_RANGE (axpy scalar), MQ_ERR_SIZE, MQ_ERR_OOM, MQ_ERR_CUDA.
 */
int mq_batch_create(mq_batch **out, const mq_job *jobs, size_t njobs, const mq_batch_opts *opts, void *stream);

/*
 * Replace the jobs' pointers and scalars with those of `jobs`, which must have the same kinds,
 * dependencies, plans' sizes and widths, lengths and batch sizes as at creation (the item table
 * is reused).  Asynchronous on `stream`: launches ordered after it on the same stream see the
 * new table.  Errors: MQ_ERR_ARG (shape differs), MQ_ERR_ALIGN, MQ_ERR_RANGE, MQ_ERR_CUDA.
 */
int mq_batch_update(mq_batch *b, const mq_job *jobs, size_t njobs, void *stream);

/* Run the batch on `stream` (replays the captured graph).  Asynchronous. */
int mq_batch_launch(mq_batch *b, void *stream);

/*
 * Wait for the last launch and return its device status: MQ_OK, MQ_ERR_TIMEOUT when a bounded
 * device-side wait gave up (the batch's results are then incomplete; the device stays usable), or
 * MQ_ERR_RANGE when the input check of a checked job failed (no job ran).
 */
int mq_batch_status(mq_batch *b);

/* Work items, persistent CTAs (0 for the calls form) and items of each kind, for reports (any pointer
   may be NULL). */
int mq_batch_info(const mq_batch *b, size_t *items, unsigned *ctas, size_t *ntt_items, size_t *blas_items);

/* Free a batch (synchronises with the device first).  NULL is accepted. */
int mq_batch_destroy(mq_batch *b);

/*
 * Autotuner: time candidate options on this batch shape with a few launches each -- the persistent
 * forms x CTAs per SM x pipeline lag x BLAS chunk, then, around the fastest, the stage fusion of
 * two-pass transforms (split_shift -1, +1) and the calls form -- write the fastest to *best and, if
 * cache_path is non-NULL, record it in that JSON cache under a key made of the device name and the
 * batch shape (each job's kind, size, width, order and dependency).  The jobs' buffers are
 * overwritten (the timing runs the batch).  Errors: those of mq_batch_create.
 */
int mq_autotune_batch(const mq_job *jobs, size_t njobs, mq_batch_opts *best, const char *cache_path, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MQNTT_BATCH_H */

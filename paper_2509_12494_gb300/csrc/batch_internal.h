// batch_internal.h -- the batched persistent form's tables and launcher, shared by the batch API
// (batch.cu) and the serving loop (serve.cu).  Internal to the library.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "../../include/mqntt_batch.h"
#include "check.h"
#include "common.cuh"

namespace mq {
namespace batch_detail {

// Transform tiles of 2^L residues per work item (one CTA of 256 threads, 2048 residues), L = 6..11.
// The kernels' tile shape must agree: batch_kernel.cuh checks it at compile time.
constexpr unsigned tiles_per_cta(int L) { return 1u << (11 - L); }

constexpr int JK_NTT = 0, JK_BLAS = 1;

struct JobDev {
    int kind;        // JK_NTT or JK_BLAS
    int width;       // 1 or 2 words per residue
    int inv;         // NTT direction
    int op;          // BLAS op (OP_*)
    int after;       // job this one waits for, or -1
    int twopass;     // NTT: two passes (per-polynomial counters)
    int L[2];        // NTT: tile log size of pass 0 and pass 1
    unsigned n_items;     // items of this job (target of its completion counter)
    unsigned poly_base;   // two-pass NTT: index of polynomial 0's counter
    unsigned groups0;     // two-pass NTT: pass-0 items per polynomial
    unsigned pad;
    unsigned long long chunk;  // BLAS: residues per item
    PassArgs pa[2];            // NTT passes
    BlasArgs ba;               // BLAS operands
    int tma[2];                // pass p takes the TMA form (tma.cuh); its tensor maps follow
    CUtensorMap tm[2][2];      // [pass][0: source, 1: destination]; 128-byte aligned by their type
};

// One work item (32 bytes; the prefetching kernel copies it into shared memory with two 16-byte
// copies).  The host resolves its dependency and completion counters, indices into the counter
// array of a launch: [0] next item, [1] status, [2, 2 + njobs) finished items per job, then
// finished first-pass items per polynomial of two-pass transforms.
struct ItemDev {
    unsigned job;
    unsigned short pass;
    unsigned short meta;  // what the kernel needs to pick its code path without reading the job
                          // descriptor: ITEM_BLAS | ITEM_W128 | ITEM_INV | ITEM_TMA | (tile log size << 4)
    unsigned poly;
    unsigned dep;     // counter this item waits for, 0: none
    unsigned target;  // value the dependency counter must reach
    unsigned bump;    // counter to add one to when done besides the job's (first passes), 0: none
    unsigned long long first;  // NTT: first tile of the pass; BLAS: chunk index
};
static_assert(sizeof(ItemDev) == 32, "work items are copied as two 16-byte halves");
constexpr unsigned ITEM_BLAS = 1, ITEM_W128 = 2, ITEM_INV = 4, ITEM_TMA = 8;
__host__ __device__ constexpr unsigned item_meta(bool blas, int width, bool inv, int L, bool tma = false) {
    return (blas ? ITEM_BLAS : 0u) | (width == 2 ? ITEM_W128 : 0u) | (inv ? ITEM_INV : 0u) | (tma ? ITEM_TMA : 0u) |
           ((unsigned)L << 4);
}

// Kernel instantiation of batches of 128-bit transforms whose every pass takes the TMA form
// (job_variant's 2 with this bit): the kernel carries only that code path.
constexpr int VARIANT_TMA_ONLY = 2 | 8;

// Host-side expansion of a job list into the device tables of one launch.
struct BatchTables {
    std::vector<JobDev> jobs;
    std::vector<ItemDev> items;
    size_t n_ctrs = 0;        // counters to zero before each launch
    size_t ntt_items = 0, blas_items = 0;
    int variant = 3;          // kernel instantiation (job_variant)
};

// Staging bytes a job needs (natural-order transforms in two passes), 0 if none.
size_t job_scratch_bytes(const mq_job &j);

// Validate `jobs`, fill `out` (job descriptors with `scratch[i]` as job i's staging, and the work
// items in pipelining order).  `grid_items` is the number of items the persistent grid holds at
// once (it scales the pipelining lag).  Returns MQ_OK or an MQ_ERR_* code (message set).
int build_tables(const mq_job *jobs, size_t njobs, const mq_batch_opts &opts, void *const *scratch,
                 unsigned long long grid_items, BatchTables &out);

// Validate one job on its own (as job 0 of a batch): MQ_OK or an MQ_ERR_* code (message set).
int check_job(const mq_job &j, const mq_batch_opts &opts);

// Re-fill the descriptors of an already built batch with new pointers / scalars (same shapes).
int refill_jobs(const mq_job *jobs, size_t njobs, const mq_batch_opts &opts, void *const *scratch,
                std::vector<JobDev> &jobs_io);

// Which persistent kernel instantiation covers the jobs: residue widths present (bit 0: 64-bit,
// bit 1: 128-bit) | 4 if any BLAS job.
int job_variant(const mq_job *jobs, size_t njobs);

// Kernel form for a batch: 0 warp-specialised, 1 prefetching (MQ_BATCH_FORM_* flags, else the
// default for the variant).
int kernel_form(int variant, unsigned flags);

// Persistent CTAs of the instantiation for `variant` and `form` with `ctas_per_sm` (0: as many as
// fit) on the current device, and the bytes of one tile buffer.
int persistent_grid(int variant, int form, unsigned ctas_per_sm, unsigned *grid, size_t *smem);

// Zero the counters, run the input check of the n_check operands in dcheck (if any; check_max is the
// largest one's residue count), and launch the persistent kernel instantiation that covers
// `variant` (the tables' variant) on `s` (asynchronous).
cudaError_t launch_persistent(int variant, int form, const JobDev *djobs, const ItemDev *ditems, unsigned n_items,
                              unsigned *dctrs, size_t n_ctrs, unsigned njobs, unsigned long long limit_ns,
                              unsigned grid, size_t smem, cudaStream_t s, const CheckRec *dcheck = nullptr,
                              unsigned n_check = 0, unsigned long long check_max = 0);

void apply_defaults(mq_batch_opts &o);

}  // namespace batch_detail
}  // namespace mq

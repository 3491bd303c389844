// batch.cu -- the batched persistent form (include/mqntt_batch.h).
//
// A batch is a list of jobs (NTT passes of plans, BLAS operations) expanded on the host into work
// items of one CTA each: a group of transform tiles (the same tile_group code as the per-call
// kernels) or a chunk of a BLAS vector.  One persistent kernel, one wave of CTAs, takes items in
// order from a device counter.  Dependencies always point to earlier items:
//   * the second pass of a two-pass transform waits for the first pass of the same polynomial
//     (a per-polynomial counter of finished first-pass items);
//   * the first items of a job with `after` wait for every item of that job (a per-job counter).
// Items are ordered by a software-pipelining key: job chains (a job and the jobs that depend on
// it) are laid out in submission order, chain c starting at position P(c) = the number of
// first-stage items of the chains before it; an item of stage s (its pass, plus the stages of the
// jobs before it in its chain) gets the key P(c) + s * D, D = lag x 2 x CTAs of the persistent
// grid (lag waves, counting two items per CTA), so a dependent stage is fetched about D items
// after its producer and its waits are normally already satisfied.  A lag of several waves
// matters because a CTA of the prefetching form takes its items up to three ahead.
// Deadlock freedom: an item waits only for items fetched before it; those were fetched by CTAs
// that are running, whose own waits are again for earlier items, so every wait ends.  Each wait
// is still bounded (globaltimer) and sets the batch status to MQ_ERR_TIMEOUT when it gives up;
// every CTA then drains out, so a broken batch never hangs the GPU.
// Memory ordering: a finished item's threads fence, the CTA synchronises, and one thread adds to
// the counters; a waiting thread reads counters with ld.acquire.gpu and the CTA synchronises
// before touching data.  Data moves through L2 (.cg loads and stores), so no SM reads a stale L1
// line of a buffer another SM rewrote during the launch.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mqntt_batch.h"
#include "batch_internal.h"
#include "trace.h"
#include "batch_kernel.cuh"
#include "blas_ops.cuh"
#include "common.cuh"
#include "hostmath.h"
#include "ntt_kernel.cuh"
#include "plan.h"

int mq_fail(int code, const char *fmt, ...);
int mq_cuda_fail(cudaError_t e, const char *where);
int mq_check_modulus(const uint64_t q[2], int width, hm::u128 *qv);

namespace mq {
namespace batch_detail {

}  // namespace batch_detail
}  // namespace mq

using namespace mq;
using namespace mq::batch_detail;

// ------------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------------

struct mq_batch {
    int device = 0;
    std::vector<mq_job> shape;
    std::vector<JobDev> hjobs;
    std::vector<void *> scratch;  // per job (natural-order two-pass transforms), else nullptr
    JobDev *djobs = nullptr;
    JobDev *pinned_jobs = nullptr;
    ItemDev *ditems = nullptr;
    unsigned *dctrs = nullptr;
    size_t n_ctrs = 0;
    size_t n_items = 0, ntt_items = 0, blas_items = 0;
    int variant = 3;  // kernel instantiation (job_variant)
    int form = 0;     // kernel form (kernel_form)
    unsigned grid = 0;
    size_t smem = 0;
    unsigned long long limit_ns = 0;
    mq_batch_opts opts{};
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr, staged = nullptr;
    int *h_status = nullptr;
    bool launched = false;
    bool calls = false;                // MQ_BATCH_FORM_CALLS: the graph holds the jobs' own kernels
    CheckRec *dcheck = nullptr;        // operands of the jobs that carry MQ_CHECK_INPUTS (device table)
    unsigned n_check = 0;
    unsigned long long check_max = 0;  // residues of the largest checked operand
};


static int job_passes(const mq_job &j) {
    if (j.kind == MQ_JOB_NTT_FORWARD || j.kind == MQ_JOB_NTT_INVERSE) return j.plan->log2n <= 11 ? 1 : 2;
    return 1;
}

static bool is_ntt(int kind) { return kind == MQ_JOB_NTT_FORWARD || kind == MQ_JOB_NTT_INVERSE; }

// The operands a launch checks before any job runs: the data of NTT jobs whose plan carries
// MQ_CHECK_INPUTS, both inputs of BLAS jobs whose width carries it (axpy: x and y).
static void check_records(const mq_job *jobs, size_t njobs, std::vector<CheckRec> &out, unsigned long long &max_res) {
    out.clear();
    max_res = 0;
    for (size_t i = 0; i < njobs; ++i) {
        const mq_job &j = jobs[i];
        if (is_ntt(j.kind)) {
            if (!(j.plan->flags & MQ_CHECK_INPUTS)) continue;
            const size_t N = (size_t)1 << j.plan->log2n, batch = j.batch ? j.batch : 1;
            out.push_back(check_rec(j.data, batch, N, batch == 1 ? N : j.stride, j.plan->width, j.plan->q, "job data"));
            max_res = std::max<unsigned long long>(max_res, (unsigned long long)batch * N);
        } else if ((unsigned)j.width & MQ_CHECK_INPUTS) {
            const int w = (int)((unsigned)j.width & ~MQ_CHECK_INPUTS);
            out.push_back(check_rec(j.a, 1, j.n, j.n, w, j.q, "job input a"));
            out.push_back(check_rec(j.kind == MQ_JOB_AXPY ? j.data : j.b, 1, j.n, j.n, w, j.q, "job input b"));
            max_res = std::max<unsigned long long>(max_res, j.n);
        }
    }
}

static int blas_op_of(int kind) {
    switch (kind) {
    case MQ_JOB_VADD: return OP_VADD;
    case MQ_JOB_VSUB: return OP_VSUB;
    case MQ_JOB_VMUL: return OP_VMUL;
    default: return OP_AXPY;
    }
}

// Validate one job and fill its device descriptor (pointers, constants).  `scr` is the job's
// staging buffer (natural-order two-pass transforms only).
static int fill_job(const mq_job &j, size_t index, const mq_batch_opts &o, void *scr, JobDev &d) {
    memset(&d, 0, sizeof d);
    if (j.after >= (int)index) return mq_fail(MQ_ERR_ARG, "job %zu: `after` must name an earlier job", index);
    if (j.after < -1) return mq_fail(MQ_ERR_ARG, "job %zu: bad `after`", index);
    d.after = j.after;
    if (is_ntt(j.kind)) {
        const ntt_plan *p = j.plan;
        if (!p) return mq_fail(MQ_ERR_ARG, "job %zu: NTT job without a plan", index);
        if (p->width > MQ_W128) return mq_fail(MQ_ERR_ARG, "job %zu: the batched form takes residues of one or two words", index);
        if (p->log2n < LMIN || p->log2n > 2 * LMAX)
            return mq_fail(MQ_ERR_SIZE, "job %zu: batched transforms need 2^%d <= N <= 2^%d", index, LMIN, 2 * LMAX);
        if (!j.data) return mq_fail(MQ_ERR_ARG, "job %zu: data is NULL", index);
        if (((uintptr_t)j.data) % 16) return mq_fail(MQ_ERR_ALIGN, "job %zu: data is not 16-byte aligned", index);
        const size_t N = (size_t)1 << p->log2n;
        const size_t batch = j.batch ? j.batch : 1;
        const size_t stride = batch == 1 ? N : j.stride;
        if (stride < N) return mq_fail(MQ_ERR_SIZE, "job %zu: stride shorter than N", index);
        const bool inv = j.kind == MQ_JOB_NTT_INVERSE;
        const bool natural = !(p->flags & MQ_ORDER_BITREV);
        const int logN = (int)p->log2n;
        d.kind = JK_NTT;
        d.width = p->width;
        d.inv = inv;
        d.twopass = logN > LMAX;
        int L1 = 0;
        if (d.twopass) {  // stage fusion: the even split moved by split_shift, both passes within LMIN..LMAX
            L1 = logN / 2 + o.split_shift;
            L1 = std::max(L1, std::max(LMIN, logN - LMAX));
            L1 = std::min(L1, std::min(LMAX, logN - LMIN));
        }
        const int L2 = logN - L1;
        for (int k = 0; k < 2; ++k) {
            PassArgs &a = d.pa[k];
            a.tw = inv ? p->tw_inv : p->tw_fwd;
            memcpy(a.q, p->q, sizeof a.q);
            memcpy(a.sc, p->sc, sizeof a.sc);
            memcpy(a.scp, p->scp, sizeof a.scp);
            memcpy(a.ws, p->ws, sizeof a.ws);
            memcpy(a.wsp, p->wsp, sizeof a.wsp);
            a.batch = batch;
            a.logN = logN;
            a.L1 = L1;
        }
        if (!d.twopass) {
            PassArgs &a = d.pa[0];
            a.in = a.out = j.data;
            a.in_stride = a.out_stride = stride;
            a.in_layout = (inv && natural) ? LAYOUT_NAT : LAYOUT_ROW;
            a.out_layout = (!inv && natural) ? LAYOUT_NAT : LAYOUT_ROW;
            a.scale = inv;
            a.final = 1;
            d.L[0] = logN;
        } else {
            PassArgs &first = d.pa[0], &second = d.pa[1];
            PassArgs &col = inv ? second : first, &row = inv ? first : second;
            col.col = 1;
            col.in_layout = col.out_layout = LAYOUT_COL;
            row.col = 0;
            row.perm = natural;
            if (!inv) {
                col.in = j.data;
                col.in_stride = stride;
                col.out = natural ? scr : j.data;
                col.out_stride = natural ? N : stride;
                row.in = col.out;
                row.in_stride = col.out_stride;
                row.out = j.data;
                row.out_stride = stride;
                row.in_layout = LAYOUT_ROW;
                row.out_layout = natural ? LAYOUT_NAT : LAYOUT_ROW;
                row.final = 1;
                d.L[0] = L1;
                d.L[1] = L2;
            } else {
                row.in = j.data;
                row.in_stride = stride;
                row.out = natural ? scr : j.data;
                row.out_stride = natural ? N : stride;
                row.in_layout = natural ? LAYOUT_NAT : LAYOUT_ROW;
                row.out_layout = LAYOUT_ROW;
                col.in = row.out;
                col.in_stride = row.out_stride;
                col.out = j.data;
                col.out_stride = stride;
                col.scale = 1;
                col.final = 1;
                d.L[0] = L2;
                d.L[1] = L1;
            }
            // passes of 128-bit tiles of 2^8 in the column or unpermuted row view take the TMA form
            for (int k = 0; k < 2; ++k) {
                const PassArgs &a = d.pa[k];
                d.tma[k] = d.width == MQ_W128 && d.L[k] == TMA_L && tma_eligible(a) &&
                           tile_map(&d.tm[k][0], a.col != 0, a.in, a.logN, a.L1, a.batch, a.in_stride) == 0 &&
                           tile_map(&d.tm[k][1], a.col != 0, a.out, a.logN, a.L1, a.batch, a.out_stride) == 0;
            }
        }
        return MQ_OK;
    }
    if (j.kind < MQ_JOB_VADD || j.kind > MQ_JOB_AXPY) return mq_fail(MQ_ERR_ARG, "job %zu: unknown kind %d", index, j.kind);
    const int width = (int)((unsigned)j.width & ~MQ_CHECK_INPUTS);  // the check flag rides on the width
    hm::u128 Q;
    int rc = mq_check_modulus(j.q, width, &Q);
    if (rc) return rc;
    if (j.n == 0) return mq_fail(MQ_ERR_ARG, "job %zu: empty vector", index);
    const void *ptrs[3] = {j.data, j.a, j.kind == MQ_JOB_AXPY ? j.data : j.b};
    for (int k = 0; k < 3; ++k) {
        if (!ptrs[k]) return mq_fail(MQ_ERR_ARG, "job %zu: NULL operand", index);
        if (((uintptr_t)ptrs[k]) % 16) return mq_fail(MQ_ERR_ALIGN, "job %zu: operands must be 16-byte aligned", index);
    }
    d.kind = JK_BLAS;
    d.width = width;
    d.op = blas_op_of(j.kind);
    d.chunk = o.blas_chunk;
    BlasArgs &b = d.ba;
    b.c = j.data;
    b.a = j.a;
    b.b = ptrs[2];
    b.n = j.n;
    memcpy(b.q, j.q, sizeof b.q);
    b.L = hm::bitlen(Q);
    hm::to_words(hm::barrett_mu(Q, b.L), b.mu);
    if (j.kind == MQ_JOB_AXPY) {
        hm::u128 s = hm::from_words(j.scalar);
        if (s >= Q || (width == MQ_W64 && j.scalar[1])) return mq_fail(MQ_ERR_RANGE, "job %zu: scalar must be < q", index);
        hm::to_words(s, b.s);
        hm::to_words(hm::shoup(s, Q, width == MQ_W64 ? 64 : 128), b.sp);
    }
    return MQ_OK;
}

static bool same_shape(const mq_job &a, const mq_job &b) {
    if (a.kind != b.kind || a.after != b.after) return false;
    if (is_ntt(a.kind)) {
        if (!b.plan || a.plan->log2n != b.plan->log2n || a.plan->width != b.plan->width ||
            (a.plan->flags & MQ_ORDER_BITREV) != (b.plan->flags & MQ_ORDER_BITREV))
            return false;
        return (a.batch ? a.batch : 1) == (b.batch ? b.batch : 1);
    }
    return a.n == b.n && a.width == b.width;
}

void mq::batch_detail::apply_defaults(mq_batch_opts &o) {
    if (o.lag == 0) o.lag = 32;  // stage-major for batches up to 32 waves per stage (see the lag sweep)
    if (o.blas_chunk == 0) o.blas_chunk = 16384;
    o.blas_chunk = (o.blas_chunk + 2047) / 2048 * 2048;
    if (o.wait_timeout_s <= 0) o.wait_timeout_s = 2.0;
}

size_t mq::batch_detail::job_scratch_bytes(const mq_job &j) {
    if (is_ntt(j.kind) && j.plan && j.plan->log2n > LMAX && j.plan->log2n <= 2 * LMAX && !(j.plan->flags & MQ_ORDER_BITREV))
        return (j.batch ? j.batch : 1) * ((size_t)1 << j.plan->log2n) * 8u * (size_t)j.plan->width;
    return 0;
}

int mq::batch_detail::refill_jobs(const mq_job *jobs, size_t njobs, const mq_batch_opts &opts, void *const *scratch,
                                  std::vector<JobDev> &io) {
    for (size_t i = 0; i < njobs; ++i) {
        JobDev d;
        int rc = fill_job(jobs[i], i, opts, scratch ? scratch[i] : nullptr, d);
        if (rc) return rc;
        d.n_items = io[i].n_items;  // counters and item bookkeeping stay those of the build
        d.poly_base = io[i].poly_base;
        d.groups0 = io[i].groups0;
        if (d.tma[0] != io[i].tma[0] || d.tma[1] != io[i].tma[1])  // the items' copy form is fixed at build
            return mq_fail(MQ_ERR_ARG, "job %zu: the update changes how its passes are staged", i);
        io[i] = d;
    }
    return MQ_OK;
}

int mq::batch_detail::check_job(const mq_job &j, const mq_batch_opts &opts) {
    JobDev d;
    return fill_job(j, 0, opts, (void *)(uintptr_t)256, d);  // stand-in staging pointer, never dereferenced
}

int mq::batch_detail::build_tables(const mq_job *jobs, size_t njobs, const mq_batch_opts &opts, void *const *scratch,
                                   unsigned long long grid_items, BatchTables &out) {
    out.jobs.assign(njobs, JobDev());
    out.items.clear();
    out.ntt_items = out.blas_items = 0;
    for (size_t i = 0; i < njobs; ++i) {
        if (job_scratch_bytes(jobs[i]) && !(scratch && scratch[i]))
            return mq_fail(MQ_ERR_ARG, "job %zu: natural-order transform without staging", i);
        int rc = fill_job(jobs[i], i, opts, scratch ? scratch[i] : nullptr, out.jobs[i]);
        if (rc) return rc;
    }
    // pipeline lag in work items: `lag` times what the persistent grid holds at once, so a
    // dependent stage is fetched well after its producer items finished
    const unsigned long long lag_items = (unsigned long long)opts.lag * grid_items;

    // expand into items, ordered by the pipelining key
    struct Key {
        unsigned long long key;
        unsigned stage, chain;
        ItemDev it;
    };
    std::vector<Key> keys;
    std::vector<unsigned> chain(njobs), depth(njobs);
    std::vector<unsigned long long> chain_pos;  // first item position of each chain, in items
    unsigned long long next_pos = 0;
    unsigned next_chain = 0, poly_ctrs = 0;
    bool dropped = !(opts.flags & MQ_BATCH_TEST_DROP_ITEM);
    long drop_job = -1;
    for (size_t i = 0; i < njobs; ++i) {
        const mq_job &j = jobs[i];
        JobDev &d = out.jobs[i];
        if (j.after < 0) {
            chain[i] = next_chain++;
            depth[i] = 0;
            chain_pos.push_back(next_pos);
        } else {
            chain[i] = chain[j.after];
            depth[i] = depth[j.after] + (unsigned)job_passes(jobs[j.after]);
        }
        unsigned count = 0;
        auto push = [&](unsigned pass, unsigned poly, unsigned long long first) {
            Key k;
            k.stage = depth[i] + pass;
            k.chain = chain[i];
            k.key = chain_pos[k.chain] + (unsigned long long)k.stage * lag_items;
            k.it.job = (unsigned)i;
            k.it.pass = (unsigned short)pass;
            k.it.meta = (unsigned short)item_meta(d.kind == JK_BLAS, d.width, d.inv != 0, d.kind == JK_NTT ? d.L[pass] : 0,
                                                  d.kind == JK_NTT && d.tma[pass] != 0);
            k.it.poly = poly;
            k.it.dep = k.it.target = k.it.bump = 0;  // resolved once every job's item count is known
            k.it.first = first;
            if (!dropped && is_ntt(j.kind) && d.twopass && pass == 0) {
                dropped = true;  // fault injection: this item never runs
                drop_job = (long)i;
            } else {
                keys.push_back(k);
                ++count;
            }
        };
        if (d.kind == JK_NTT) {
            const unsigned long long batch = d.pa[0].batch;
            if (!d.twopass) {
                const unsigned G = tiles_per_cta(d.L[0]);
                for (unsigned long long t = 0; t < batch; t += G) push(0, 0, t);
                out.ntt_items += (batch + G - 1) / G;
            } else {
                d.poly_base = poly_ctrs;
                poly_ctrs += (unsigned)batch;
                for (int pass = 0; pass < 2; ++pass) {
                    const PassArgs &a = d.pa[pass];
                    const unsigned TP = a.col ? (1u << (a.logN - a.L1)) : (1u << a.L1);
                    const unsigned G = tiles_per_cta(d.L[pass]);
                    const unsigned groups = TP / G;
                    if (pass == 0) d.groups0 = groups;
                    for (unsigned long long p = 0; p < batch; ++p)
                        for (unsigned g = 0; g < groups; ++g) push(pass, (unsigned)p, p * TP + (unsigned long long)g * G);
                    out.ntt_items += batch * groups;
                }
            }
        } else {
            const unsigned long long chunks = (d.ba.n + d.chunk - 1) / d.chunk;
            for (unsigned long long c = 0; c < chunks; ++c) push(0, 0, c);
            out.blas_items += chunks;
        }
        d.n_items = count;
        if (j.after < 0) next_pos += count;  // chains are spaced by the items of their first job
        if (keys.size() > 0xffffffffull) return mq_fail(MQ_ERR_SIZE, "more than 2^32 work items");
    }
    // a dropped item still counts toward its job's target: nothing can complete that job
    if (drop_job >= 0) out.jobs[drop_job].n_items += 1;
    std::stable_sort(keys.begin(), keys.end(), [](const Key &x, const Key &y) {
        if (x.key != y.key) return x.key < y.key;
        if (x.stage != y.stage) return x.stage < y.stage;
        return x.chain < y.chain;
    });
    out.items.resize(keys.size());
    const unsigned poly0 = 2 + (unsigned)njobs;  // first per-polynomial counter
    for (size_t k = 0; k < keys.size(); ++k) {
        ItemDev &it = out.items[k];
        it = keys[k].it;
        const JobDev &d = out.jobs[it.job];
        if (d.kind == JK_NTT && d.twopass && it.pass == 1) {  // the polynomial's first pass
            it.dep = poly0 + d.poly_base + it.poly;
            it.target = d.groups0;
        } else if (it.pass == 0 && d.after >= 0) {  // every item of the job it comes after
            it.dep = 2 + (unsigned)d.after;
            it.target = out.jobs[d.after].n_items;
        }
        if (d.kind == JK_NTT && d.twopass && it.pass == 0) it.bump = poly0 + d.poly_base + it.poly;
    }
    out.n_ctrs = 2 + njobs + poly_ctrs;
    out.variant = job_variant(jobs, njobs);
    if (out.variant == 2) {  // 128-bit transforms only: all of them in the TMA form?
        bool all = njobs > 0;
        for (const JobDev &d : out.jobs) all = all && d.kind == JK_NTT && d.twopass && d.tma[0] && d.tma[1];
        if (all) out.variant = VARIANT_TMA_ONLY;
    }
    return MQ_OK;
}

// the instantiations: 0 the general one (any mix), 1 64-bit transforms only, 2 128-bit transforms
// only, 3 128-bit transforms whose every pass takes the TMA form (only that code path compiled)
static int kernel_slot(int variant) {
    return variant == 1 ? 1 : variant == 2 ? 2 : variant == VARIANT_TMA_ONLY ? 3 : 0;
}

int mq::batch_detail::job_variant(const mq_job *jobs, size_t njobs) {
    int v = 0;
    for (size_t i = 0; i < njobs; ++i) {
        const bool ntt = is_ntt(jobs[i].kind);
        const int w = ntt ? (jobs[i].plan ? jobs[i].plan->width : 2) : (int)((unsigned)jobs[i].width & ~MQ_CHECK_INPUTS);
        v |= (w == MQ_W64 ? 1 : 2) | (ntt ? 0 : 4);
    }
    return v ? v : 3;
}

int mq::batch_detail::kernel_form(int variant, unsigned flags) {
    if (flags & MQ_BATCH_FORM_PREFETCH) return 1;
    if (flags & MQ_BATCH_FORM_SPLIT) return 0;
    (void)variant;  // the prefetching form measured faster for every instantiation
    return 1;
}

int mq::batch_detail::persistent_grid(int variant, int form, unsigned ctas_per_sm, unsigned *grid, size_t *smem) {
    // every instantiation gets its shared-memory limit and occupancy once per process
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    static int per_sm[2][4] = {};
    static size_t buf[2][4] = {};
    static const int max_ctas[2][4] = {
        {PersistentKernel<0, 3, true>::MAXB, PersistentKernel<0, 1, false>::MAXB, PersistentKernel<0, 2, false>::MAXB,
         PersistentKernel<0, 6, false>::MAXB},
        {PersistentKernel<1, 3, true>::MAXB, PersistentKernel<1, 1, false>::MAXB, PersistentKernel<1, 2, false>::MAXB,
         PersistentKernel<1, 6, false>::MAXB}};
    std::call_once(attr_once, [&] {
        cudaError_t e[8] = {PersistentKernel<0, 3, true>::configure(&per_sm[0][0], &buf[0][0]),
                            PersistentKernel<0, 1, false>::configure(&per_sm[0][1], &buf[0][1]),
                            PersistentKernel<0, 2, false>::configure(&per_sm[0][2], &buf[0][2]),
                            PersistentKernel<0, 6, false>::configure(&per_sm[0][3], &buf[0][3]),
                            PersistentKernel<1, 3, true>::configure(&per_sm[1][0], &buf[1][0]),
                            PersistentKernel<1, 1, false>::configure(&per_sm[1][1], &buf[1][1]),
                            PersistentKernel<1, 2, false>::configure(&per_sm[1][2], &buf[1][2]),
                            PersistentKernel<1, 6, false>::configure(&per_sm[1][3], &buf[1][3])};
        for (cudaError_t x : e)
            if (x != cudaSuccess && attr_err == cudaSuccess) attr_err = x;
    });
    const int k = kernel_slot(variant), f = form ? 1 : 0;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (attr_err != cudaSuccess || per_sm[f][k] < 1)
        return mq_fail(MQ_ERR_CUDA, "the persistent kernel does not fit on an SM");
    const unsigned fit = std::min<unsigned>((unsigned)per_sm[f][k], (unsigned)max_ctas[f][k]);
    *grid = (unsigned)sms * (ctas_per_sm ? std::min(ctas_per_sm, fit) : fit);
    *smem = buf[f][k];
    return MQ_OK;
}

cudaError_t mq::batch_detail::launch_persistent(int variant, int form, const JobDev *djobs, const ItemDev *ditems,
                                                unsigned n_items, unsigned *dctrs, size_t n_ctrs, unsigned njobs,
                                                unsigned long long limit_ns, unsigned grid, size_t smem,
                                                cudaStream_t s, const CheckRec *dcheck, unsigned n_check,
                                                unsigned long long check_max) {
    cudaError_t e = cudaMemsetAsync(dctrs, 0, n_ctrs * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    if (n_check) {  // a failed input check ends the item counter, so no job runs
        e = launch_batch_check(dcheck, n_check, check_max, dctrs, n_items, s);
        if (e != cudaSuccess) return e;
    }
    const int k = kernel_slot(variant);
#define MQ_LAUNCH(F, WM, BL) return PersistentKernel<F, WM, BL>::launch(djobs, ditems, n_items, dctrs, njobs, limit_ns, grid, smem, s)
    if (form) {
        if (k == 3) MQ_LAUNCH(1, 6, false);
        if (k == 2) MQ_LAUNCH(1, 2, false);
        if (k == 1) MQ_LAUNCH(1, 1, false);
        MQ_LAUNCH(1, 3, true);
    }
    if (k == 3) MQ_LAUNCH(0, 6, false);
    if (k == 2) MQ_LAUNCH(0, 2, false);
    if (k == 1) MQ_LAUNCH(0, 1, false);
    MQ_LAUNCH(0, 3, true);
#undef MQ_LAUNCH
}

static int lookup_tuned(const std::vector<mq_job> &jobs, mq_batch_opts &o);

static void destroy_batch(mq_batch *b) {
    if (!b) return;
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cs) cudaStreamDestroy(b->cs);
    if (b->done) cudaEventDestroy(b->done);
    if (b->staged) cudaEventDestroy(b->staged);
    if (b->h_status) cudaFreeHost(b->h_status);
    if (b->pinned_jobs) cudaFreeHost(b->pinned_jobs);
    if (b->djobs) cudaFree(b->djobs);
    if (b->ditems) cudaFree(b->ditems);
    if (b->dctrs) cudaFree(b->dctrs);
    if (b->dcheck) cudaFree(b->dcheck);
    for (void *p : b->scratch)
        if (p) cudaFree(p);
    delete b;
}

// The calls form of one job: the kernels the per-call entry points launch for it (transform passes
// with the batch's pass split and staging, or the BLAS kernel), on `s`.
static cudaError_t launch_job_calls(const JobDev &d, cudaStream_t s) {
    if (d.kind == JK_NTT) {
        cudaError_t e = launch_ntt_pass(d.width, d.L[0], d.inv != 0, d.pa[0], s);
        if (e == cudaSuccess && d.twopass) e = launch_ntt_pass(d.width, d.L[1], d.inv != 0, d.pa[1], s);
        return e;
    }
    return launch_blas(d.width, d.op, d.ba, s);
}

static int enqueue_run(mq_batch *b, cudaStream_t s) {
    if (b->calls) {  // every job's kernels in job order: an earlier job always finishes first.  Nothing
                     // waits on the device, so there are no counters to reset and the status stays MQ_OK.
        cudaError_t e = cudaSuccess;
        for (size_t i = 0; i < b->hjobs.size() && e == cudaSuccess; ++i) e = launch_job_calls(b->hjobs[i], s);
        return e == cudaSuccess ? MQ_OK : mq_cuda_fail(e, "batch launch (calls form)");
    }
    cudaError_t e = launch_persistent(b->variant, b->form, b->djobs, b->ditems, (unsigned)b->n_items, b->dctrs, b->n_ctrs,
                                      (unsigned)b->hjobs.size(), b->limit_ns, b->grid, b->smem, s, b->dcheck, b->n_check,
                                      b->check_max);
    if (e != cudaSuccess) return mq_cuda_fail(e, "persistent kernel launch");
    e = cudaMemcpyAsync(b->h_status, b->dctrs + 1, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return mq_cuda_fail(e, "status copy");
    return MQ_OK;
}

// Capture one launch (enqueue_run) on the batch's stream into a graph, instantiate and upload it.
// A graph captured before is destroyed first (the calls form captures its jobs' pointers, so an
// update re-captures).
static int capture_graph(mq_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return mq_cuda_fail(e, "graph capture");
    int rc = enqueue_run(b, b->cs);
    cudaError_t e2 = cudaStreamEndCapture(b->cs, &b->graph);
    if (rc) return rc;
    if (e2 != cudaSuccess) return mq_cuda_fail(e2, "graph capture");
    if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess) return mq_cuda_fail(e, "graph instantiate");
    // upload now, so that the first launch does not pay for it on the caller's stream
    if ((e = cudaGraphUpload(b->exec, b->cs)) != cudaSuccess || (e = cudaStreamSynchronize(b->cs)) != cudaSuccess)
        return mq_cuda_fail(e, "graph upload");
    return MQ_OK;
}

extern "C" int mq_batch_create(mq_batch **out, const mq_job *jobs, size_t njobs, const mq_batch_opts *opts, void *stream) {
    MQ_TRACE("mq_batch_create");
    if (!out) return mq_fail(MQ_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!jobs || njobs == 0) return mq_fail(MQ_ERR_ARG, "a batch needs at least one job");
    if (njobs > (1u << 24)) return mq_fail(MQ_ERR_ARG, "too many jobs");
    mq_batch *b = new mq_batch();
    cudaGetDevice(&b->device);
    b->shape.assign(jobs, jobs + njobs);
    if (opts) {
        b->opts = *opts;
    } else {
        lookup_tuned(b->shape, b->opts);
    }
    apply_defaults(b->opts);
    b->limit_ns = (unsigned long long)(b->opts.wait_timeout_s * 1e9);
    b->scratch.assign(njobs, nullptr);
    b->variant = job_variant(jobs, njobs);
    b->form = kernel_form(b->variant, b->opts.flags);
    int rc = persistent_grid(b->variant, b->form, b->opts.ctas_per_sm, &b->grid, &b->smem);
    if (rc) {
        destroy_batch(b);
        return rc;
    }
    // staging for natural-order two-pass transforms
    for (size_t i = 0; i < njobs; ++i) {
        const size_t bytes = job_scratch_bytes(jobs[i]);
        if (!bytes) continue;
        cudaError_t e = cudaMalloc(&b->scratch[i], bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            destroy_batch(b);
            return mq_fail(MQ_ERR_OOM, "job %zu: staging of %zu bytes does not fit", i, bytes);
        }
    }
    BatchTables t;
    rc = build_tables(jobs, njobs, b->opts, b->scratch.data(), 2ull * b->grid, t);
    if (!rc && t.variant != b->variant) {  // the TMA-only instantiation (same grid and buffers)
        b->variant = t.variant;
        rc = persistent_grid(b->variant, b->form, b->opts.ctas_per_sm, &b->grid, &b->smem);
    }
    if (rc) {
        destroy_batch(b);
        return rc;
    }
    b->hjobs = std::move(t.jobs);
    b->n_items = t.items.size();
    b->n_ctrs = t.n_ctrs;
    b->ntt_items = t.ntt_items;
    b->blas_items = t.blas_items;

    cudaError_t e;
    if ((e = cudaMalloc(&b->djobs, njobs * sizeof(JobDev))) != cudaSuccess ||
        (e = cudaMalloc(&b->ditems, std::max<size_t>(1, t.items.size()) * sizeof(ItemDev))) != cudaSuccess ||
        (e = cudaMalloc(&b->dctrs, b->n_ctrs * sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMallocHost(&b->pinned_jobs, njobs * sizeof(JobDev))) != cudaSuccess ||
        (e = cudaMallocHost(&b->h_status, sizeof(int))) != cudaSuccess) {
        cudaGetLastError();
        destroy_batch(b);
        return mq_fail(MQ_ERR_OOM, "batch tables do not fit");
    }
    *b->h_status = 0;
    cudaStream_t s = (cudaStream_t)stream;
    memcpy(b->pinned_jobs, b->hjobs.data(), njobs * sizeof(JobDev));
    if ((e = cudaMemcpyAsync(b->djobs, b->pinned_jobs, njobs * sizeof(JobDev), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(b->ditems, t.items.data(), t.items.size() * sizeof(ItemDev), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
        destroy_batch(b);
        return mq_cuda_fail(e, "batch table upload");
    }
    {
        std::vector<CheckRec> recs;
        check_records(jobs, njobs, recs, b->check_max);
        if (!recs.empty()) {
            if ((e = cudaMalloc(&b->dcheck, recs.size() * sizeof(CheckRec))) != cudaSuccess) {
                cudaGetLastError();
                destroy_batch(b);
                return mq_fail(MQ_ERR_OOM, "input check table does not fit");
            }
            if ((e = cudaMemcpy(b->dcheck, recs.data(), recs.size() * sizeof(CheckRec), cudaMemcpyHostToDevice)) !=
                cudaSuccess) {
                destroy_batch(b);
                return mq_cuda_fail(e, "input check table upload");
            }
            b->n_check = (unsigned)recs.size();
        }
    }
    {
        // the calls form: asked for, or the default when a persistent grid would mostly idle
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
        const unsigned forms = b->opts.flags & (MQ_BATCH_FORM_SPLIT | MQ_BATCH_FORM_PREFETCH | MQ_BATCH_FORM_CALLS);
        if ((forms & MQ_BATCH_FORM_CALLS) && b->n_check) {
            destroy_batch(b);
            return mq_fail(MQ_ERR_ARG, "the calls form does not run the input check of checked jobs");
        }
        b->calls = (forms & MQ_BATCH_FORM_CALLS) || (!forms && !b->n_check && b->n_items < (size_t)sms);
        // a persistent grid of no more CTAs than there are items
        b->grid = (unsigned)std::min<size_t>(b->grid, std::max<size_t>(1, b->n_items));
    }
    if ((e = cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming)) != cudaSuccess) {
        destroy_batch(b);
        return mq_cuda_fail(e, "batch stream/events");
    }
    if (!(b->opts.flags & MQ_BATCH_NO_GRAPH) && (rc = capture_graph(b))) {
        destroy_batch(b);
        return rc;
    }
    *out = b;
    return MQ_OK;
}

extern "C" int mq_batch_update(mq_batch *b, const mq_job *jobs, size_t njobs, void *stream) {
    MQ_TRACE("mq_batch_update");
    if (!b || !jobs) return mq_fail(MQ_ERR_ARG, "NULL batch or jobs");
    if (njobs != b->shape.size()) return mq_fail(MQ_ERR_ARG, "the batch has %zu jobs, got %zu", b->shape.size(), njobs);
    for (size_t i = 0; i < njobs; ++i)
        if (!same_shape(b->shape[i], jobs[i])) return mq_fail(MQ_ERR_ARG, "job %zu differs in shape from the batch's", i);
    std::vector<JobDev> next = b->hjobs;
    int rc = refill_jobs(jobs, njobs, b->opts, b->scratch.data(), next);
    if (rc) return rc;
    cudaError_t e = cudaEventSynchronize(b->staged);  // the previous upload has left the staging buffer
    if (e != cudaSuccess) return mq_cuda_fail(e, "staging wait");
    b->hjobs = next;
    memcpy(b->pinned_jobs, b->hjobs.data(), njobs * sizeof(JobDev));
    cudaStream_t s = (cudaStream_t)stream;
    if ((e = cudaMemcpyAsync(b->djobs, b->pinned_jobs, njobs * sizeof(JobDev), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaEventRecord(b->staged, s)) != cudaSuccess)
        return mq_cuda_fail(e, "job table upload");
    if (b->n_check) {  // same shapes, so the same operands are checked: only their pointers change
        std::vector<CheckRec> recs;
        unsigned long long mx = 0;
        check_records(jobs, njobs, recs, mx);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess ||
            (e = cudaMemcpy(b->dcheck, recs.data(), recs.size() * sizeof(CheckRec), cudaMemcpyHostToDevice)) != cudaSuccess)
            return mq_cuda_fail(e, "input check table upload");
    }
    for (size_t i = 0; i < njobs; ++i) b->shape[i] = jobs[i];
    if (b->calls && b->exec) {  // the graph holds the old pointers: capture it again once it is idle
        if (b->launched && (e = cudaEventSynchronize(b->done)) != cudaSuccess) return mq_cuda_fail(e, "batch wait");
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return mq_cuda_fail(e, "job table upload");
        return capture_graph(b);
    }
    return MQ_OK;
}

extern "C" int mq_batch_launch(mq_batch *b, void *stream) {
    MQ_TRACE("mq_batch_launch");
    if (!b) return mq_fail(MQ_ERR_ARG, "batch is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (b->exec) {
        e = cudaGraphLaunch(b->exec, s);
        if (e != cudaSuccess) return mq_cuda_fail(e, "graph launch");
    } else {
        int rc = enqueue_run(b, s);
        if (rc) return rc;
    }
    e = cudaEventRecord(b->done, s);
    if (e != cudaSuccess) return mq_cuda_fail(e, "event record");
    b->launched = true;
    return MQ_OK;
}

extern "C" int mq_batch_status(mq_batch *b) {
    if (!b) return mq_fail(MQ_ERR_ARG, "batch is NULL");
    if (!b->launched) return MQ_OK;
    cudaError_t e = cudaEventSynchronize(b->done);
    if (e != cudaSuccess) return mq_cuda_fail(e, "batch wait");
    int st = *(volatile int *)b->h_status;
    if (st == MQ_ERR_RANGE) return mq_fail(st, "an input residue of a checked job is not below q: no job of the batch ran");
    if (st != 0) return mq_fail(st, "a device-side wait of the batch gave up after %.3f s", b->opts.wait_timeout_s);
    return MQ_OK;
}

extern "C" int mq_batch_info(const mq_batch *b, size_t *items, unsigned *ctas, size_t *ntt_items, size_t *blas_items) {
    if (!b) return mq_fail(MQ_ERR_ARG, "batch is NULL");
    if (items) *items = b->n_items;
    if (ctas) *ctas = b->calls ? 0u : b->grid;
    if (ntt_items) *ntt_items = b->ntt_items;
    if (blas_items) *blas_items = b->blas_items;
    return MQ_OK;
}

extern "C" int mq_batch_destroy(mq_batch *b) {
    destroy_batch(b);
    return MQ_OK;
}

// ------------------------------------------------------------------------------------------------
// autotuner
// ------------------------------------------------------------------------------------------------

static uint64_t fnv1a(const std::string &s) {
    uint64_t h = 1469598103934665603ull;
    for (unsigned char c : s) {
        h ^= c;
        h *= 1099511628211ull;
    }
    return h;
}

// Key: device name and the batch shape (kinds, sizes, widths, dependencies), hashed.
static std::string shape_key(const std::vector<mq_job> &jobs) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    memset(&prop, 0, sizeof prop);
    cudaGetDeviceProperties(&prop, dev);
    std::string sig;
    char buf[96];
    for (const mq_job &j : jobs) {
        if (is_ntt(j.kind))
            snprintf(buf, sizeof buf, "%d:%u:%d:%u:%zu:%d;", j.kind, j.plan ? j.plan->log2n : 0, j.plan ? j.plan->width : 0,
                     j.plan ? j.plan->flags : 0, j.batch, j.after);
        else
            snprintf(buf, sizeof buf, "%d:%zu:%d:%d;", j.kind, j.n, j.width, j.after);
        sig += buf;
    }
    char key[160];
    snprintf(key, sizeof key, "%s|%zu|%016llx", prop.name, jobs.size(), (unsigned long long)fnv1a(sig));
    for (char *c = key; *c; ++c)
        if (*c == '"' || *c == '\\') *c = '_';
    return key;
}

static std::string read_file(const char *path) {
    std::string s;
    FILE *f = fopen(path, "rb");
    if (!f) return s;
    char buf[4096];
    size_t n;
    while ((n = fread(buf, 1, sizeof buf, f)) > 0) s.append(buf, n);
    fclose(f);
    return s;
}

// The cache is a JSON object of "key": {"ctas_per_sm": c, "lag": l, "blas_chunk": b, "form": f, "split": s,
// "ms": t} with f = 0 (warp-specialised), 1 (prefetching) or 2 (calls).
static bool cache_get(const char *path, const std::string &key, mq_batch_opts &o) {
    std::string s = read_file(path);
    size_t at = s.find("\"" + key + "\"");
    if (at == std::string::npos) return false;
    unsigned c = 0, l = 0, bc = 0, form = 1;
    int split = 0;
    const int got = sscanf(s.c_str() + at + key.size() + 2,
                           " : {\"ctas_per_sm\": %u, \"lag\": %u, \"blas_chunk\": %u, \"form\": %u, \"split\": %d", &c,
                           &l, &bc, &form, &split);
    if (got < 3) return false;
    o.ctas_per_sm = c;
    o.lag = l;
    o.blas_chunk = bc;
    o.split_shift = split;
    o.flags = (o.flags & ~(MQ_BATCH_FORM_SPLIT | MQ_BATCH_FORM_PREFETCH | MQ_BATCH_FORM_CALLS)) |
              (form == 2 ? MQ_BATCH_FORM_CALLS : form ? MQ_BATCH_FORM_PREFETCH : MQ_BATCH_FORM_SPLIT);
    return true;
}

static void cache_put(const char *path, const std::string &key, const mq_batch_opts &o, double ms) {
    std::string s = read_file(path);
    std::vector<std::string> entries;
    // keep every other entry: one per line between the braces
    size_t pos = 0;
    while ((pos = s.find("\n  \"", pos)) != std::string::npos) {
        size_t end = s.find('}', pos);
        if (end == std::string::npos) break;
        std::string line = s.substr(pos + 3, end + 1 - (pos + 3));
        if (line.compare(0, key.size() + 2, "\"" + key + "\"") != 0) entries.push_back(line);
        pos = end;
    }
    char buf[512];
    const int form = (o.flags & MQ_BATCH_FORM_CALLS) ? 2 : (o.flags & MQ_BATCH_FORM_SPLIT) ? 0 : 1;
    snprintf(buf, sizeof buf,
             "\"%s\": {\"ctas_per_sm\": %u, \"lag\": %u, \"blas_chunk\": %u, \"form\": %d, \"split\": %d, \"ms\": %.4f}",
             key.c_str(), o.ctas_per_sm, o.lag, o.blas_chunk, form, o.split_shift, ms);
    entries.push_back(buf);
    std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "wb");
    if (!f) return;
    fputs("{", f);
    for (size_t i = 0; i < entries.size(); ++i) fprintf(f, "%s\n  %s", i ? "," : "", entries[i].c_str());
    fputs("\n}\n", f);
    fclose(f);
    rename(tmp.c_str(), path);
}

static int lookup_tuned(const std::vector<mq_job> &jobs, mq_batch_opts &o) {
    const char *path = getenv("MQNTT_TUNE_CACHE");
    if (!path || !*path) return 0;
    return cache_get(path, shape_key(jobs), o) ? 1 : 0;
}

extern "C" int mq_autotune_batch(const mq_job *jobs, size_t njobs, mq_batch_opts *best, const char *cache_path, void *stream) {
    MQ_TRACE("mq_autotune_batch");
    if (!jobs || !njobs || !best) return mq_fail(MQ_ERR_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    bool has_blas = false, has_deps = false, has_twopass = false, has_check = false;
    for (size_t i = 0; i < njobs; ++i) {
        const bool ntt = is_ntt(jobs[i].kind);
        has_blas |= !ntt;
        has_twopass |= ntt && jobs[i].plan && jobs[i].plan->log2n > LMAX;
        has_deps |= jobs[i].after >= 0 || (ntt && jobs[i].plan && jobs[i].plan->log2n > LMAX);
        has_check |= ntt ? (jobs[i].plan && (jobs[i].plan->flags & MQ_CHECK_INPUTS)) : (((unsigned)jobs[i].width & MQ_CHECK_INPUTS) != 0);
    }
    const unsigned forms[] = {MQ_BATCH_FORM_PREFETCH, MQ_BATCH_FORM_SPLIT};
    const unsigned ctas[] = {1, 2, 3, 4};  // beyond what an instantiation holds, the grid repeats and is skipped
    const unsigned lags[] = {1, 2, 4, 8, 16, 32};
    const unsigned chunks[] = {8192, 16384, 65536};
    double best_ms = 1e30;
    mq_batch_opts bo{};
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    // mean event time of 5 launches after 2 warm-ups; keeps the fastest in bo / best_ms
    auto trial = [&](const mq_batch_opts &o) -> int {
        mq_batch *b = nullptr;
        int rc = mq_batch_create(&b, jobs, njobs, &o, stream);
        if (rc) return rc;
        float ms = 0, sum = 0;
        for (int r = 0; r < 2; ++r) mq_batch_launch(b, stream);
        for (int r = 0; r < 5; ++r) {
            cudaEventRecord(t0, s);
            mq_batch_launch(b, stream);
            cudaEventRecord(t1, s);
            cudaEventSynchronize(t1);
            cudaEventElapsedTime(&ms, t0, t1);
            sum += ms;
        }
        rc = mq_batch_status(b);
        mq_batch_destroy(b);
        if (rc) return rc;
        if (sum / 5 < best_ms) {
            best_ms = sum / 5;
            bo = o;
        }
        return MQ_OK;
    };
    int rc = MQ_OK;
    // 1. the persistent forms x CTAs per SM x lag x BLAS chunk
    for (unsigned fm : forms) {
        unsigned last_grid = 0;
        for (unsigned c : ctas) {
            unsigned grid = 0;
            size_t smem = 0;
            rc = persistent_grid(job_variant(jobs, njobs), fm == MQ_BATCH_FORM_PREFETCH, c, &grid, &smem);
            if (rc) goto done;
            if (grid == last_grid) continue;  // more CTAs per SM than this instantiation holds
            last_grid = grid;
            for (unsigned l : lags) {
                if (!has_deps && l != 2) continue;
                for (unsigned ch : chunks) {
                    if (!has_blas && ch != 16384) continue;
                    mq_batch_opts o{};
                    o.ctas_per_sm = c;
                    o.lag = l;
                    o.blas_chunk = ch;
                    o.flags = fm;
                    if ((rc = trial(o))) goto done;
                }
            }
        }
    }
    // 2. around the fastest: the stage fusion of two-pass transforms, then the calls form
    if (has_twopass) {
        const mq_batch_opts base = bo;
        for (int sh : {-1, 1}) {
            mq_batch_opts o = base;
            o.split_shift = sh;
            if ((rc = trial(o))) goto done;
        }
    }
    if (!has_check) {
        mq_batch_opts o = bo;
        o.flags = (o.flags & ~(MQ_BATCH_FORM_SPLIT | MQ_BATCH_FORM_PREFETCH)) | MQ_BATCH_FORM_CALLS;
        if ((rc = trial(o))) goto done;
    }
    *best = bo;
    apply_defaults(*best);
    if (cache_path && *cache_path) cache_put(cache_path, shape_key(std::vector<mq_job>(jobs, jobs + njobs)), *best, best_ms);
done:
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    return rc;
}

// batch_kernel.cuh -- the warp-specialised persistent kernel of the batched form, as a template
// over the residue widths and job kinds it carries (instantiated in batch_k_*.cu).
#pragma once
#include <cuda_runtime.h>

#include "batch_internal.h"
#include "blas_ops.cuh"
#include "common.cuh"
#include "ntt_kernel.cuh"

namespace mq {
namespace batch_detail {

using ntt_detail::Shape;
using ntt_detail::Traits;

constexpr int BT = 256;               // threads per persistent CTA
constexpr int LMIN = 6, LMAX = 11;    // tile sizes the persistent kernel carries

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Add one to a completion counter with release semantics at GPU scope: the writes that precede it
// (this thread's, and cumulatively those ordered before it by a barrier) are visible to any thread
// that acquires the counter and sees the increment.  No return value, so the thread does not wait
// for the addition itself.
__device__ __forceinline__ void red_release_add(unsigned *p) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(p) : "memory");
}

__device__ __forceinline__ int ld_status(const unsigned *p) {
    return (int)*(const volatile unsigned *)p;
}

// Bounded wait until *ctr >= target.  Returns false on timeout or when the batch already failed.
static __device__ __noinline__ bool wait_geq(const unsigned *ctr, unsigned target, const unsigned *status, unsigned long long limit_ns) {
    if (ld_acquire(ctr) >= target) return true;
    const unsigned long long t0 = globaltimer();
    for (;;) {
        __nanosleep(200);
        if (ld_acquire(ctr) >= target) return true;
        if (ld_status(status) != 0) return false;
        if (globaltimer() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ uint4 u4(const uint64_t v[2]) {
    return make_uint4((uint32_t)v[0], (uint32_t)(v[0] >> 32), (uint32_t)v[1], (uint32_t)(v[1] >> 32));
}

// residues [begin, end) of a BLAS job; 16-byte aligned operands (checked on the host)
template <int W, int OP>
__device__ __forceinline__ void blas_chunk(const BlasArgs &b, unsigned long long begin, unsigned long long end, int tid) {
    if (W == 2) {
        const Mod128 m{u4(b.q), u4(b.mu), b.L};
        const uint4 s = u4(b.s), sp = u4(b.sp);
        const uint4 *A = reinterpret_cast<const uint4 *>(b.a), *B = reinterpret_cast<const uint4 *>(b.b);
        uint4 *C = reinterpret_cast<uint4 *>(b.c);
        // one residue per thread and step: the wave of resident CTAs keeps enough loads in flight,
        // and an unrolled Barrett would spill inside this many-branched kernel
        for (unsigned long long i = begin + tid; i < end; i += BT) {
            const uint4 va = __ldcg(A + i), vb = __ldcg(B + i);
            __stcg(C + i, op128<OP>(va, vb, m, s, sp));
        }
    } else {
        const Mod64 m{b.q[0], b.mu[0], b.L};
        const uint64_t s = b.s[0], sp = b.sp[0];
        // begin is a multiple of the (even) chunk: pairs first, then a possible odd last residue
        const ulonglong2 *A = reinterpret_cast<const ulonglong2 *>(b.a), *B = reinterpret_cast<const ulonglong2 *>(b.b);
        ulonglong2 *C = reinterpret_cast<ulonglong2 *>(b.c);
        const unsigned long long vb0 = begin / 2, ve = end / 2;
        for (unsigned long long i = vb0 + tid; i < ve; i += BT) {
            ulonglong2 x = __ldcg(A + i), y = __ldcg(B + i), r;
            r.x = op64<OP>(x.x, y.x, m, s, sp);
            r.y = op64<OP>(x.y, y.y, m, s, sp);
            __stcg(C + i, r);
        }
        if ((end & 1) && tid == 0) {
            const unsigned long long *a1 = reinterpret_cast<const unsigned long long *>(b.a);
            const unsigned long long *b1 = reinterpret_cast<const unsigned long long *>(b.b);
            unsigned long long *c1 = reinterpret_cast<unsigned long long *>(b.c);
            c1[end - 1] = op64<OP>(__ldcg(a1 + end - 1), __ldcg(b1 + end - 1), m, s, sp);
        }
    }
}

template <int W>
__device__ __forceinline__ void run_blas(int op, const BlasArgs &b, unsigned long long begin, unsigned long long end, int tid) {
    switch (op) {
    case OP_VADD: blas_chunk<W, OP_VADD>(b, begin, end, tid); break;
    case OP_VSUB: blas_chunk<W, OP_VSUB>(b, begin, end, tid); break;
    case OP_VMUL: blas_chunk<W, OP_VMUL>(b, begin, end, tid); break;
    default: blas_chunk<W, OP_AXPY>(b, begin, end, tid); break;
    }
}

constexpr int PT = 64;              // producer threads (two warps)
constexpr int CT = BT + PT;         // threads per persistent CTA
constexpr int BAR_COMPUTE = 1;      // named barrier of the BT compute threads
constexpr int BAR_FULL = 2;         // + buffer: producer -> compute, "buffer b holds item k"
constexpr int BAR_EMPTY = 4;        // + buffer: compute -> producer, "buffer b is free again"
constexpr int BAR_PRODUCER = 6;     // named barrier of the PT producer threads

// named barriers with immediate ids (a register id would make ptxas reserve all sixteen)
__device__ __forceinline__ void bar_arrive(int id) {
    if (id == BAR_FULL) asm volatile("bar.arrive %0, %1;" ::"n"(BAR_FULL), "n"(CT) : "memory");
    else if (id == BAR_FULL + 1) asm volatile("bar.arrive %0, %1;" ::"n"(BAR_FULL + 1), "n"(CT) : "memory");
    else if (id == BAR_EMPTY) asm volatile("bar.arrive %0, %1;" ::"n"(BAR_EMPTY), "n"(CT) : "memory");
    else asm volatile("bar.arrive %0, %1;" ::"n"(BAR_EMPTY + 1), "n"(CT) : "memory");
}
__device__ __forceinline__ void bar_sync(int id) {
    if (id == BAR_FULL) asm volatile("bar.sync %0, %1;" ::"n"(BAR_FULL), "n"(CT) : "memory");
    else if (id == BAR_FULL + 1) asm volatile("bar.sync %0, %1;" ::"n"(BAR_FULL + 1), "n"(CT) : "memory");
    else if (id == BAR_EMPTY) asm volatile("bar.sync %0, %1;" ::"n"(BAR_EMPTY), "n"(CT) : "memory");
    else asm volatile("bar.sync %0, %1;" ::"n"(BAR_EMPTY + 1), "n"(CT) : "memory");
}

// Stage an item's tiles: cp.async for 128-bit residues (16-byte copies through L2).  64-bit
// residues take 8-byte copies, which also allocate in the SM's L1; those are used only where
// ASYNC64 is set, by the prefetching form, whose every dependency is taken with an acquire load
// at GPU scope before the copies start (an acquire orders the later weak loads of the CTA after
// the producer's release whatever their cache operator, so no stale L1 line can be read).  The
// split form stages 64-bit tiles with batched L2 loads.
template <int W, int NTH = PT, bool ASYNC64 = false>
__device__ __forceinline__ void stage_tiles(int L, const PassArgs &a, unsigned long long first, void *sm, int lane) {
    typedef typename Traits<W>::E E;
    E *s = reinterpret_cast<E *>(sm);
#define MQ_STAGE(LL)                                                                      \
    if (W == 2 || ASYNC64) ntt_detail::load_tiles_async<W, LL, NTH>(a, first, s, lane);   \
    else ntt_detail::load_tiles_sync<W, LL, NTH>(a, first, s, lane);                       \
    break;
    switch (L) {
    case 6: MQ_STAGE(6)
    case 7: MQ_STAGE(7)
    case 8: MQ_STAGE(8)
    case 9: MQ_STAGE(9)
    case 10: MQ_STAGE(10)
    default: MQ_STAGE(11)
    }
#undef MQ_STAGE
}

template <int W, bool INV>
__device__ __forceinline__ void compute_store(int L, const PassArgs &a, unsigned long long first, void *sm, int tid) {
    typedef typename Traits<W>::E E;
    E *s = reinterpret_cast<E *>(sm);
    switch (L) {
    case 6: ntt_detail::tile_compute_store<W, 6, INV, BAR_COMPUTE>(a, first, s, tid); break;
    case 7: ntt_detail::tile_compute_store<W, 7, INV, BAR_COMPUTE>(a, first, s, tid); break;
    case 8: ntt_detail::tile_compute_store<W, 8, INV, BAR_COMPUTE>(a, first, s, tid); break;
    case 9: ntt_detail::tile_compute_store<W, 9, INV, BAR_COMPUTE>(a, first, s, tid); break;
    case 10: ntt_detail::tile_compute_store<W, 10, INV, BAR_COMPUTE>(a, first, s, tid); break;
    default: ntt_detail::tile_compute_store<W, 11, INV, BAR_COMPUTE>(a, first, s, tid); break;
    }
}

// ctrs: [0] next item, [1] status, [2, 2 + njobs) per-job finished items, then per-polynomial
// finished first-pass items of two-pass transforms.
//
// Warp-specialised: warps 8-9 are the producer.  For item k it waits until buffer k % 2 is free,
// takes the next item index, waits (bounded) for the item's dependencies, copies its arguments
// and stages its tiles into the buffer, and hands it over.  Warps 0-7 compute and store the item,
// publish its completion on the counters, and free the buffer.  The producer therefore runs one
// item ahead, and its waits and loads overlap the transform of the previous item.
// WM: residue widths present (bit 0: 64-bit, bit 1: 128-bit; bit 2: 128-bit transforms whose every
// item is a TMA item, prefetching form); BL: BLAS jobs present.  A batch runs
// the narrowest instantiation that covers its jobs, which keeps registers and code small.  64-bit
// transforms alone need fewer registers and half the shared memory, and their arithmetic has
// shorter dependency chains per residue, so that instantiation runs one CTA per SM more (three in
// the split form, four in the prefetching form) to keep more warps in flight.
template <int WM, bool BL>
struct KCfg {
    static constexpr int MINB = (WM == 1 && !BL) ? 3 : 2;  // resident CTAs per SM the registers allow
    static constexpr int PMINB = (WM == 1 && !BL) ? 4 : 3; // the same for the prefetching form
    static constexpr int W = (WM & 2) ? 2 : 1;              // widest residue (sizes the tile buffers)
};

template <int WM, bool BL>
__global__ void __launch_bounds__(CT, KCfg<WM, BL>::MINB)
    persistent_kernel(const JobDev *__restrict__ jobs, const ItemDev *__restrict__ items, unsigned n_items,
                      unsigned *ctrs, unsigned njobs, unsigned long long limit_ns, size_t buf_bytes) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ PassArgs s_pa[2];
    __shared__ BlasArgs s_ba[2];
    __shared__ unsigned s_it[2];
    __shared__ unsigned s_pit;
    __shared__ int s_pok;
    const int tid = threadIdx.x;
    unsigned *status = ctrs + 1, *job_ctr = ctrs + 2, *poly_ctr = ctrs + 2 + njobs;

    if (tid >= BT) {  // ----------------------------------------------- producer warps
        const int lane = tid - BT;  // 0 .. PT-1
        for (unsigned k = 0;; ++k) {
            const int b = k & 1;
            if (k >= 2) bar_sync(BAR_EMPTY + b);
            if (lane == 0) {
                unsigned it0 = atomicAdd(ctrs, 1u);
                if (ld_status(status) != 0) it0 = n_items;  // the batch failed: drain
                int w = it0 < n_items;
                if (w) {
                    const ItemDev i0 = items[it0];
                    const JobDev *J0 = jobs + i0.job;
                    if (J0->kind == JK_NTT && J0->twopass && i0.pass == 1)
                        w = wait_geq(poly_ctr + J0->poly_base + i0.poly, J0->groups0, status, limit_ns);
                    else if (i0.pass == 0 && J0->after >= 0)
                        w = wait_geq(job_ctr + J0->after, jobs[J0->after].n_items, status, limit_ns);
                    if (!w) atomicCAS(status, 0u, (unsigned)MQ_ERR_TIMEOUT);
                }
                s_pit = it0;
                s_pok = w;
            }
            asm volatile("bar.sync %0, %1;" ::"n"(BAR_PRODUCER), "n"(PT) : "memory");
            const unsigned it = s_pit;
            const bool ok = s_pok != 0;
            asm volatile("bar.sync %0, %1;" ::"n"(BAR_PRODUCER), "n"(PT) : "memory");  // s_pit reusable
            ItemDev item;
            const JobDev *J = jobs;
            if (ok) {
                item = items[it];
                J = jobs + item.job;
            }
            if (!ok) {  // end of the work (or a failed wait): tell the compute warps and stop
                if (lane == 0) s_it[b] = n_items;
                __threadfence_block();
                bar_arrive(BAR_FULL + b);
                break;
            }
            if (!BL || J->kind == JK_NTT) {
                const unsigned *src = reinterpret_cast<const unsigned *>(&J->pa[item.pass]);
                unsigned *dst = reinterpret_cast<unsigned *>(&s_pa[b]);
                for (int w = lane; w < (int)(sizeof(PassArgs) / 4); w += PT) dst[w] = src[w];
                unsigned char *buf = smem_raw + b * buf_bytes;
                if ((WM & 1) && (!(WM & 2) || J->width == 1))
                    stage_tiles<1>(J->L[item.pass], J->pa[item.pass], item.first, buf, lane);
                else if (WM & 2)
                    stage_tiles<2>(J->L[item.pass], J->pa[item.pass], item.first, buf, lane);
                asm volatile("cp.async.wait_all;" ::: "memory");
            } else {
                const unsigned *src = reinterpret_cast<const unsigned *>(&J->ba);
                unsigned *dst = reinterpret_cast<unsigned *>(&s_ba[b]);
                for (int w = lane; w < (int)(sizeof(BlasArgs) / 4); w += PT) dst[w] = src[w];
            }
            if (lane == 0) s_it[b] = it;
            __threadfence_block();
            bar_arrive(BAR_FULL + b);
        }
        return;
    }

    // ------------------------------------------------------------------- compute warps
    for (unsigned k = 0;; ++k) {
        const int b = k & 1;
        bar_sync(BAR_FULL + b);
        const unsigned it = s_it[b];
        if (it >= n_items) break;
        const ItemDev item = items[it];
        const JobDev *J = jobs + item.job;
        const int kind = J->kind;
        unsigned char *buf = smem_raw + b * buf_bytes;
        if (!BL || kind == JK_NTT) {
            const int L = J->L[item.pass];
            if ((WM & 1) && (!(WM & 2) || J->width == 1)) {
                if (J->inv) compute_store<1, true>(L, s_pa[b], item.first, buf, tid);
                else compute_store<1, false>(L, s_pa[b], item.first, buf, tid);
            } else if (WM & 2) {
                if (J->inv) compute_store<2, true>(L, s_pa[b], item.first, buf, tid);
                else compute_store<2, false>(L, s_pa[b], item.first, buf, tid);
            }
        } else if (BL) {
            const BlasArgs &ba = s_ba[b];
            const unsigned long long begin = item.first * J->chunk;
            const unsigned long long end = begin + J->chunk < ba.n ? begin + J->chunk : ba.n;
            if ((WM & 1) && (!(WM & 2) || J->width == 1)) run_blas<1>(J->op, ba, begin, end, tid);
            else if (WM & 2) run_blas<2>(J->op, ba, begin, end, tid);
            ntt_detail::tile_sync<BAR_COMPUTE, BT>();
        }
        // every compute thread's stores precede the barrier above; thread 0's release makes them
        // visible (cumulatively) to whoever acquires the counters
        if (tid == 0) {
            __threadfence();
            if ((!BL || kind == JK_NTT) && J->twopass && item.pass == 0) atomicAdd(poly_ctr + J->poly_base + item.poly, 1u);
            atomicAdd(job_ctr + item.job, 1u);
        }
        __threadfence_block();
        bar_arrive(BAR_EMPTY + b);
    }
}

// Copy a work item's record into shared memory (two 16-byte copies through L2).
__device__ __forceinline__ void copy_record(ItemDev *dst, const ItemDev *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + 16), "l"(reinterpret_cast<const char *>(src) + 16)
                 : "memory");
}

// The prefetching form: all BT threads compute, and each CTA prefetches its next item while it
// transforms the current one (the per-call pass kernel's double buffering, with items from the
// work list).  No warps are set aside for staging, so every thread keeps the register budget of
// the per-call kernel (three CTAs per SM, four for 64-bit transforms alone).
//
// Thread 0 runs the item bookkeeping ahead of the transform so that its memory round trips
// overlap the arithmetic: while item k is transformed it already holds the index of item k + 3
// (an atomicAdd issued one item earlier) and has the record of item k + 2 on its way into
// shared memory.  Before item k's transform it checks, without waiting, whether item k + 1's
// dependency counter has reached its target; if so the CTA starts item k + 1's copies before the
// transform, else after it, once a bounded wait ended.  Items a CTA takes are processed in the
// order taken and depend only on items taken before them, so every wait ends (the unfinished
// item of lowest index always has its dependencies done and its CTA working on it).
template <int WM, bool BL>
__global__ void __launch_bounds__(BT, KCfg<WM, BL>::PMINB)
    prefetch_kernel(const JobDev *__restrict__ jobs, const ItemDev *__restrict__ items, unsigned n_items,
                    unsigned *ctrs, unsigned njobs, unsigned long long limit_ns, size_t buf_bytes) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ PassArgs s_pa[2];
    __shared__ BlasArgs s_ba[2];
    __shared__ __align__(8) uint64_t s_bar[2];  // tensor copies into buffer 0 / 1 (TMA items)
    __shared__ __align__(16) ItemDev s_rec[3];  // records of items k, k + 1, k + 2 (slot k % 3)
    __shared__ unsigned s_idx[3];               // their indices (n_items: none)
    // whether item k + 1's dependency was met when item k started, by the parity of k: thread 0 writes
    // item k + 1's flag before the first barrier of item k + 1, while slower threads may still be
    // reading item k's at the end of item k, so the two must not share a word
    __shared__ int s_ready[2];
    const int tid = threadIdx.x;
    unsigned *status = ctrs + 1;
    (void)njobs;
    // Instantiations with 128-bit transforms carry TMA items (ITEM_TMA): their buffers start on a
    // 1024-byte boundary (the 128-byte swizzle's period), buf_bytes apart, a multiple of 1024.
    constexpr bool TMA = (WM & 2) != 0;
    constexpr bool TMA_ONLY = (WM & 4) != 0;  // every item is a TMA item: only that path is compiled
    unsigned char *const smem = TMA ? smem_raw + ((1024u - (tma::su32(smem_raw) & 1023u)) & 1023u) : smem_raw;
    unsigned ph0 = 0, ph1 = 0;  // all threads: phase parity of the next tensor copy into buffer 0 / 1
    if (TMA && tid == 0) {
        tma::mbar_init(&s_bar[0], 1);
        tma::mbar_init(&s_bar[1], 1);
        tma::mbar_init_fence();
    }

    // all threads: copy the item's arguments and start staging its tiles into buffer b (a TMA item:
    // thread 0 issues its tensor copy, after the dependency it acquired)
    auto stage = [&](int b, const ItemDev &item) {
        const JobDev *J = jobs + item.job;
        const unsigned m = item.meta;  // kind, width and tile size without a read of the job descriptor
        if (!BL || !(m & ITEM_BLAS)) {
            const PassArgs &pa = J->pa[item.pass];
            const unsigned *src = reinterpret_cast<const unsigned *>(&pa);
            unsigned *dst = reinterpret_cast<unsigned *>(&s_pa[b]);
            for (int w = tid; w < (int)(sizeof(PassArgs) / 4); w += BT) dst[w] = src[w];
            unsigned char *buf = smem + b * buf_bytes;
            if (TMA_ONLY || (TMA && (m & ITEM_TMA))) {
                if (tid == 0) {
                    int x, y, z;
                    ntt_detail::tma_box(ntt_detail::TileAddr(pa), pa.col != 0, item.first, x, y, z);
                    tma::fence_async_global();
                    tma::mbar_expect(&s_bar[b], ntt_detail::TMA_GROUP_BYTES);
                    tma::load3(buf, &J->tm[item.pass][0], x, y, z, &s_bar[b]);
                }
            } else if ((WM & 1) && (!(WM & 2) || !(m & ITEM_W128)))
                stage_tiles<1, BT, true>((int)(m >> 4), pa, item.first, buf, tid);
            else if (WM & 2)
                stage_tiles<2, BT>((int)(m >> 4), pa, item.first, buf, tid);
        } else {
            const unsigned *src = reinterpret_cast<const unsigned *>(&J->ba);
            unsigned *dst = reinterpret_cast<unsigned *>(&s_ba[b]);
            for (int w = tid; w < (int)(sizeof(BlasArgs) / 4); w += BT) dst[w] = src[w];
        }
    };
    // thread 0: bounded wait for the dependency of the item in slot r; on timeout it is dropped
    auto wait_for = [&](int r) {
        const ItemDev &it = s_rec[r];
        if (it.dep && !wait_geq(ctrs + it.dep, it.target, status, limit_ns)) {
            atomicCAS(status, 0u, (unsigned)MQ_ERR_TIMEOUT);
            s_idx[r] = n_items;
        }
    };

    unsigned pend = 0;  // thread 0: index of the item after the two whose records are in flight
    unsigned pend_bump = 0, pend_job = 0;  // thread 0: completion counters not yet incremented (0: none)
    bool pend_tma = false;                 // thread 0: that item's results leave by a tensor store
    auto signal_pending = [&]() {
        if (pend_tma) {  // the store has landed, and is ordered before the release below
            tma::store_wait();
            tma::fence_async_global();
            pend_tma = false;
        }
        if (pend_bump) red_release_add(ctrs + pend_bump);
        if (pend_job) red_release_add(ctrs + pend_job);
        pend_bump = pend_job = 0;
    };
    if (tid == 0) {
        const unsigned i0 = atomicAdd(ctrs, 1u), i1 = atomicAdd(ctrs, 1u);
        pend = atomicAdd(ctrs, 1u);
        s_idx[0] = i0 < n_items ? i0 : n_items;
        s_idx[1] = i1 < n_items ? i1 : n_items;
        if (i0 < n_items) copy_record(&s_rec[0], items + i0);
        if (i1 < n_items) copy_record(&s_rec[1], items + i1);
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_all;" ::: "memory");
        if (i0 < n_items) wait_for(0);
    }
    __syncthreads();
    if (s_idx[0] < n_items) stage(0, s_rec[0]);
    asm volatile("cp.async.commit_group;" ::: "memory");

    for (unsigned k = 0;; ++k) {
        const int b = k & 1, r = k % 3, r1 = (k + 1) % 3, r2 = (k + 2) % 3;
        if (s_idx[r] >= n_items) break;
        if (tid == 0) {
            asm volatile("cp.async.wait_all;" ::: "memory");  // the record of item k + 1
            if (TMA) tma::store_wait_read();  // item k - 1's tensor store has read buffer b ^ 1
            int ready = 1;
            if (s_idx[r1] < n_items && s_rec[r1].dep) ready = ld_acquire(ctrs + s_rec[r1].dep) >= s_rec[r1].target;
            s_ready[b] = ready;
        }
        __syncthreads();  // s_ready[b], and the record of item k + 1
        bool early = s_idx[r1] < n_items && s_ready[b];
        if (early) stage(b ^ 1, s_rec[r1]);
        asm volatile("cp.async.commit_group;" ::: "memory");
        if (early) asm volatile("cp.async.wait_group 1;" ::: "memory");
        else asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();  // every thread's copies of the current item (and its arguments) landed
        if (tid == 0) {   // the previous item's completion, the record of item k + 2, the index of item k + 3
            if (!pend_tma) signal_pending();  // (one that left by a tensor store: at the end of this item)
            const unsigned i2 = pend < n_items ? pend : n_items;
            s_idx[r2] = i2;
            if (i2 < n_items) copy_record(&s_rec[r2], items + i2);
            asm volatile("cp.async.commit_group;" ::: "memory");
            pend = atomicAdd(ctrs, 1u);
        }

        const ItemDev &item = s_rec[r];
        const unsigned m = item.meta;
        unsigned char *buf = smem + b * buf_bytes;
        const bool tma_item = TMA_ONLY || (TMA && (m & ITEM_TMA));
        if (tma_item) {
            // every thread waits (bounded) for the tensor copy; on a timeout it marks the batch
            // failed and goes on, so that no barrier is left unmatched
            if (!tma::mbar_wait(&s_bar[b], b ? ph1 : ph0, limit_ns)) atomicCAS(status, 0u, (unsigned)MQ_ERR_TIMEOUT);
            if (b) ph1 ^= 1u;
            else ph0 ^= 1u;
            const PassArgs &pa = s_pa[b];
            uint4 *tb = reinterpret_cast<uint4 *>(buf);
            if (m & ITEM_INV) {
                if (pa.col) ntt_detail::tma_rounds<true, true>(pa, tb, item.first, tid);
                else ntt_detail::tma_rounds<true, false>(pa, tb, item.first, tid);
            } else {
                if (pa.col) ntt_detail::tma_rounds<false, true>(pa, tb, item.first, tid);
                else ntt_detail::tma_rounds<false, false>(pa, tb, item.first, tid);
            }
            tma::fence_async_shared();
            __syncthreads();
            if (tid == 0) {
                int x, y, z;
                ntt_detail::tma_box(ntt_detail::TileAddr(pa), pa.col != 0, item.first, x, y, z);
                tma::store3(&jobs[item.job].tm[item.pass][1], x, y, z, tb);
                tma::store_commit();
            }
        } else if (!BL || !(m & ITEM_BLAS)) {
            const int L = (int)(m >> 4);
            if ((WM & 1) && (!(WM & 2) || !(m & ITEM_W128))) {
                if (m & ITEM_INV) compute_store<1, true>(L, s_pa[b], item.first, buf, tid);
                else compute_store<1, false>(L, s_pa[b], item.first, buf, tid);
            } else if (WM & 2) {
                if (m & ITEM_INV) compute_store<2, true>(L, s_pa[b], item.first, buf, tid);
                else compute_store<2, false>(L, s_pa[b], item.first, buf, tid);
            }
        } else if (BL) {
            const JobDev *J = jobs + item.job;
            const BlasArgs &ba = s_ba[b];
            const unsigned long long begin = item.first * J->chunk;
            const unsigned long long end = begin + J->chunk < ba.n ? begin + J->chunk : ba.n;
            if ((WM & 1) && (!(WM & 2) || J->width == 1)) run_blas<1>(J->op, ba, begin, end, tid);
            else if (WM & 2) run_blas<2>(J->op, ba, begin, end, tid);
            ntt_detail::tile_sync<BAR_COMPUTE, BT>();
        }
        // every thread's stores precede the barrier that ends the item; thread 0's release additions
        // make them visible (cumulatively) to whoever acquires the counters.  When the next item is
        // already staged, the additions wait until that item's copies have landed (below, after the
        // second barrier of the next iteration), so that their latency overlaps the next transform
        // instead of holding every warp at the next barrier -- or, for an item whose results leave
        // by a tensor store, until the end of the next item, once that store has landed; before any
        // wait of this CTA they are made at once (after the store), so no wait can depend on an
        // addition this CTA has not made yet.
        if (TMA && !tma_item) tma::fence_async_shared();  // before a later tensor copy into this buffer
        if (tid == 0) {
            // The previous item's results, if they left by a tensor store, are released here, an
            // item after that store was issued, so that it has landed and the wait costs nothing;
            // this item's store (if any) stays in flight.
            if (pend_tma) {
                if (tma_item) tma::store_wait_all_but_last();
                else tma::store_wait();
                tma::fence_async_global();
                pend_tma = false;
                signal_pending();
            }
            pend_bump = item.bump;
            pend_job = 2 + item.job;
            pend_tma = tma_item;
        }
        // re-read from shared memory rather than keep registers live across the transform
        // (s_ready[b] changes only at item k + 2's start, s_idx[r1] only in the late path below)
        early = s_ready[b];
        if (s_idx[(k + 1) % 3] < n_items && !early) {  // the next item was not ready: wait for it now, then stage it
            const int q1 = (k + 1) % 3;
            if (tid == 0) {
                signal_pending();
                wait_for(q1);
            }
            __syncthreads();
            if (s_idx[q1] < n_items) stage((k & 1) ^ 1, s_rec[q1]);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
    }
    if (tid == 0) {
        signal_pending();  // the last item's completion
        if (TMA) tma::store_wait();
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// The host expands transform passes into items of tiles_per_cta(L) tiles: the tile shape the kernels
// use must hold exactly that many tiles on the 256 threads of a CTA.
template <int W, int L>
constexpr bool group_matches_items() {
    return Shape<W, L>::G == tiles_per_cta(L) && Shape<W, L>::NT == 256;
}
static_assert(group_matches_items<1, 6>() && group_matches_items<1, 7>() && group_matches_items<1, 8>() &&
                  group_matches_items<1, 9>() && group_matches_items<1, 10>() && group_matches_items<1, 11>(),
              "64-bit tile groups differ from the host's work items");
static_assert(group_matches_items<2, 6>() && group_matches_items<2, 7>() && group_matches_items<2, 8>() &&
                  group_matches_items<2, 9>() && group_matches_items<2, 10>() && group_matches_items<2, 11>(),
              "128-bit tile groups differ from the host's work items");

// Shared memory of one buffer: the largest tile group of width W (every group holds 2048 residues).
template <int W>
inline size_t kernel_smem() {
    size_t m = 0;
    m = m > Shape<W, 6>::SMEM ? m : Shape<W, 6>::SMEM;
    m = m > Shape<W, 7>::SMEM ? m : Shape<W, 7>::SMEM;
    m = m > Shape<W, 8>::SMEM ? m : Shape<W, 8>::SMEM;
    m = m > Shape<W, 9>::SMEM ? m : Shape<W, 9>::SMEM;
    m = m > Shape<W, 10>::SMEM ? m : Shape<W, 10>::SMEM;
    m = m > Shape<W, 11>::SMEM ? m : Shape<W, 11>::SMEM;
    return (m + 15) / 16 * 16;
}

// Launch helpers of one instantiation (defined in batch_k_*.cu).  FORM 0: warp-specialised
// (persistent_kernel), FORM 1: prefetching (prefetch_kernel).
template <int FORM, int WM, bool BL>
struct PersistentKernel {
    static constexpr int THREADS = FORM ? BT : CT;
    static constexpr int MAXB = FORM ? KCfg<WM, BL>::PMINB : KCfg<WM, BL>::MINB;  // CTAs per SM the registers allow
    // set the shared-memory limit; *per_sm = resident CTAs per SM, *smem = bytes of one buffer
    static cudaError_t configure(int *per_sm, size_t *smem);
    static cudaError_t launch(const JobDev *djobs, const ItemDev *ditems, unsigned n_items, unsigned *dctrs,
                              unsigned njobs, unsigned long long limit_ns, unsigned grid, size_t smem, cudaStream_t s);
};

// Bytes of one buffer and of the dynamic shared memory: the prefetching form with 128-bit
// transforms rounds its buffers up to 1024-byte multiples and adds 1024 bytes to align the first
// (TMA items, tma.cuh).
template <int FORM, int W>
constexpr size_t buffer_bytes(size_t tiles) {
    return (FORM && W == 2) ? ((tiles > ntt_detail::TMA_GROUP_BYTES ? tiles : ntt_detail::TMA_GROUP_BYTES) + 1023) / 1024 * 1024
                            : tiles;
}
template <int FORM, int W>
constexpr size_t dynamic_bytes(size_t buf) {
    return (FORM && W == 2) ? 2 * buf + 1024 : 2 * buf;
}

#define MQ_DEFINE_PERSISTENT_FORM(FORM, KERNEL, WM, BL)                                                   \
    template <>                                                                                            \
    cudaError_t PersistentKernel<FORM, WM, BL>::configure(int *per_sm, size_t *smem) {                     \
        constexpr int W_ = KCfg<WM, BL>::W;                                                                \
        *smem = buffer_bytes<FORM, W_>(kernel_smem<W_>());                                                 \
        const size_t dyn = dynamic_bytes<FORM, W_>(*smem);                                                 \
        cudaError_t e = cudaFuncSetAttribute(KERNEL<WM, BL>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                             (int)dyn);                                                    \
        if (e != cudaSuccess) return e;                                                                    \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, KERNEL<WM, BL>, THREADS, dyn);        \
    }                                                                                                      \
    template <>                                                                                            \
    cudaError_t PersistentKernel<FORM, WM, BL>::launch(const JobDev *djobs, const ItemDev *ditems, unsigned n_items, \
                                                       unsigned *dctrs, unsigned njobs, unsigned long long limit_ns, \
                                                       unsigned grid, size_t smem, cudaStream_t s) {           \
        const size_t dyn = dynamic_bytes<FORM, KCfg<WM, BL>::W>(smem);                                     \
        KERNEL<WM, BL><<<grid, THREADS, dyn, s>>>(djobs, ditems, n_items, dctrs, njobs, limit_ns, smem);   \
        return cudaGetLastError();                                                                         \
    }

#define MQ_DEFINE_PERSISTENT(WM, BL)                          \
    MQ_DEFINE_PERSISTENT_FORM(0, persistent_kernel, WM, BL)   \
    MQ_DEFINE_PERSISTENT_FORM(1, prefetch_kernel, WM, BL)

}  // namespace batch_detail
}  // namespace mq

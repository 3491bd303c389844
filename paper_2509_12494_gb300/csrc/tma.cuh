// tma.cuh -- tensor-memory-accelerator (TMA) tile copies and the mbarriers that track them.
//
// A pass stages a group of 2048 residues (32 KiB of 128-bit residues) per CTA.  With TMA one
// thread issues the whole group as a single tensor copy (cp.async.bulk.tensor) that lands in
// shared memory with the 128-byte swizzle -- 16-byte granule c of 128-byte row r at c ^ (r & 7),
// the layout the register rounds already use (swz<2>) -- and completes on an mbarrier, and the
// transformed group goes back to global memory the same way.  The threads issue no per-residue
// copies, and the copy engine does the column pass' strided gather and scatter.
//
// Two views of a batch of N = N1 x N2 transforms (see tile_map in ntt.cu):
//   column view: words of a row of the N1 x N2 matrix, rows, polynomials; a box of 16 words x
//     2^L1 rows holds element l of 8 adjacent columns in its 128-byte row l: shared layout
//     [l][c ^ (l & 7)];
//   row view: 128-byte rows of the polynomial, polynomials; a box of 16 words x 256 rows holds 8
//     consecutive rows (tiles) of 2^8 residues: shared layout [g][swz<2>(l)], tiles of 4 KiB.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mq {
namespace tma {

__device__ __forceinline__ unsigned su32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
// make the initialised barriers visible to the copy engine
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// one arrival that also announces `bytes` of copies completing on the barrier
__device__ __forceinline__ void mbar_expect(uint64_t *b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}

// whether the phase of parity `parity` has completed
__device__ __forceinline__ bool mbar_test(uint64_t *b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait until the phase completes or `limit_ns` pass; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, unsigned parity, unsigned long long limit_ns) {
    if (mbar_test(b, parity)) return true;
    const unsigned long long t0 = now_ns();
    for (;;) {
        if (mbar_test(b, parity)) return true;
        if (now_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void prefetch_map(const CUtensorMap *m) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(m) : "memory");
}

// Tensor copy of the box at (x, y, z) into shared memory, completing on `bar`.  x counts 8-byte
// words and is always a multiple of 2 here (16-byte aligned starts).
__device__ __forceinline__ void load3(void *dst, const CUtensorMap *m, int x, int y, int z, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            su32(dst)),
        "l"(m), "r"(x), "r"(y), "r"(z), "r"(su32(bar))
        : "memory");
}

// Tensor copy of shared memory to the box at (x, y, z), in the thread's current bulk group.
__device__ __forceinline__ void store3(const CUtensorMap *m, int x, int y, int z, const void *src) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(m), "r"(x),
                 "r"(y), "r"(z), "r"(su32(src))
                 : "memory");
}
__device__ __forceinline__ void store_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the thread's committed stores have finished reading shared memory
__device__ __forceinline__ void store_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// the thread's committed stores are complete
__device__ __forceinline__ void store_wait() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// ... all but the most recently committed one
__device__ __forceinline__ void store_wait_all_but_last() { asm volatile("cp.async.bulk.wait_group 1;" ::: "memory"); }

// Order this thread's ordinary shared-memory accesses before later copy-engine accesses.
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// ... and its global-memory accesses (an acquired dependency) before later copy-engine reads.
__device__ __forceinline__ void fence_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

}  // namespace tma
}  // namespace mq

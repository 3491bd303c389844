// check.cu -- the input range check of MQ_CHECK_INPUTS: every residue an operation reads must be
// canonical, 0 <= x < q (the precondition of Sec. 2.1 for the operands of the modular operations,
// and of the transform's coefficients).  The check only reads: it compares each residue's words
// with q's from the top word down and records the lowest index of a failing operand.
#include <cuda_runtime.h>
#include <string.h>

#include "check.h"

int mq_fail(int code, const char *fmt, ...);
int mq_cuda_fail(cudaError_t e, const char *where);
int mq_pool_alloc(void **p, size_t bytes, cudaStream_t s);
int mq_pool_free(void *p, cudaStream_t s);

namespace mq {
namespace {

constexpr int CHECK_THREADS = 256;

// x < q for a residue of W words at p (low word first)
template <int W>
__device__ __forceinline__ bool canonical(const unsigned long long *p, const uint64_t *q) {
#pragma unroll
    for (int k = W - 1; k >= 0; --k) {
        const unsigned long long x = __ldcg(p + k);
        if (x != q[k]) return x < q[k];
    }
    return false;  // x == q
}

// Residues i of operand r (grid-stride over its polys x n residues); true if one is not canonical.
template <int W>
__device__ bool any_bad(const CheckRec &r, unsigned long long i0, unsigned long long step) {
    const unsigned long long total = r.polys * r.n;
    const unsigned long long *base = reinterpret_cast<const unsigned long long *>(r.p);
    for (unsigned long long i = i0; i < total; i += step) {
        const unsigned long long poly = i / r.n, j = i - poly * r.n;
        if (!canonical<W>(base + (poly * r.stride + j) * W, r.q)) return true;
    }
    return false;
}

__device__ __forceinline__ bool rec_bad(const CheckRec &r, unsigned long long i0, unsigned long long step) {
    switch (r.width) {
    case 1: return any_bad<1>(r, i0, step);
    case 2: return any_bad<2>(r, i0, step);
    case 3: return any_bad<3>(r, i0, step);
    default: return any_bad<4>(r, i0, step);
    }
}

// One operand per launch (the per-call entry points): *bad <- min(*bad, index) on failure.
__global__ void __launch_bounds__(CHECK_THREADS) check_one_kernel(const CheckRec r, unsigned index, unsigned *bad) {
    const unsigned long long t = (unsigned long long)blockIdx.x * CHECK_THREADS + threadIdx.x;
    if (rec_bad(r, t, (unsigned long long)gridDim.x * CHECK_THREADS)) atomicMin(bad, index);
}

// Every checked operand of a batch (blockIdx.y = operand).  On failure the batch's status word
// becomes MQ_ERR_RANGE and its item counter jumps to the end, so that the persistent kernel that
// follows takes no item and no job of the batch runs.
__global__ void __launch_bounds__(CHECK_THREADS)
    check_batch_kernel(const CheckRec *recs, unsigned nrec, unsigned *ctrs, unsigned n_items) {
    const unsigned long long t = (unsigned long long)blockIdx.x * CHECK_THREADS + threadIdx.x;
    for (unsigned k = blockIdx.y; k < nrec; k += gridDim.y) {
        if (rec_bad(recs[k], t, (unsigned long long)gridDim.x * CHECK_THREADS)) {
            atomicCAS(ctrs + 1, 0u, (unsigned)MQ_ERR_RANGE);
            atomicMax(ctrs, n_items);
            return;
        }
    }
}

unsigned check_blocks() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (unsigned)(sms > 0 ? sms : 1) * 8u;  // 8 CTAs of 256 threads per SM: one full wave
}

}  // namespace

CheckRec check_rec(const void *p, unsigned long long polys, unsigned long long n, unsigned long long stride, int width,
                   const uint64_t *q, const char *name) {
    CheckRec r;
    memset(&r, 0, sizeof r);
    r.p = p;
    r.polys = polys;
    r.n = n;
    r.stride = polys > 1 ? stride : n;
    r.width = width;
    memcpy(r.q, q, sizeof(uint64_t) * (size_t)(width < 2 ? 2 : width));
    if (width == 1) r.q[1] = 0;
    r.name = name;
    return r;
}

int range_check(const CheckRec *recs, int nrec, cudaStream_t s) {
    if (nrec <= 0) return MQ_OK;
    unsigned *d_bad = nullptr;
    int rc = mq_pool_alloc((void **)&d_bad, sizeof(unsigned), s);
    if (rc) return rc;
    unsigned h_bad = ~0u;
    cudaError_t e = cudaMemsetAsync(d_bad, 0xff, sizeof(unsigned), s);
    const unsigned blocks = check_blocks();
    for (int i = 0; i < nrec && e == cudaSuccess; ++i) {
        const unsigned long long total = recs[i].polys * recs[i].n;
        if (total == 0) continue;
        const unsigned long long need = (total + CHECK_THREADS - 1) / CHECK_THREADS;
        check_one_kernel<<<(unsigned)(need < blocks ? need : blocks), CHECK_THREADS, 0, s>>>(recs[i], (unsigned)i, d_bad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_bad, d_bad, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    const int rc2 = mq_pool_free(d_bad, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return mq_cuda_fail(e, "input range check");
    if (rc2) return rc2;
    if (h_bad < (unsigned)nrec) return mq_fail(MQ_ERR_RANGE, "%s holds a residue that is not below q", recs[h_bad].name);
    return MQ_OK;
}

cudaError_t launch_batch_check(const CheckRec *d_recs, unsigned nrec, unsigned long long max_residues, unsigned *dctrs,
                               unsigned n_items, cudaStream_t s) {
    if (nrec == 0) return cudaSuccess;
    const unsigned blocks = check_blocks();
    const unsigned long long need = (max_residues + CHECK_THREADS - 1) / CHECK_THREADS;
    const unsigned gx = (unsigned)(need < 1 ? 1 : (need < blocks ? need : blocks));
    const unsigned gy = nrec < 65535u ? nrec : 65535u;
    check_batch_kernel<<<dim3(gx, gy), CHECK_THREADS, 0, s>>>(d_recs, nrec, dctrs, n_items);
    return cudaGetLastError();
}

}  // namespace mq

// noalloc.cu -- ntt_forward_noalloc: the forward transform with no device allocation at all.
//
// ntt_forward stages natural-order transforms above 2^12 residues through a buffer taken from a
// stream-ordered memory pool.  Callers that must not allocate device memory once they are running
// -- services that reserve a fixed memory budget at start-up, code that shares the device with a
// framework whose allocator owns all free memory, code recorded into a CUDA graph that may not
// contain allocation nodes -- use this entry point instead.  Its staging buffer is the file-scope
// device array below, so the call itself never allocates or frees.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "../../include/mqntt.h"
#include "common.cuh"
#include "plan.h"
#include "trace.h"

int mq_fail(int code, const char *fmt, ...);
int mq_cuda_fail(cudaError_t e, const char *where);
int mq_check_ptr(const void *p, int width, const char *name);  // the alignment rule of every entry point

using namespace mq;

// The staging buffer.  Every device that loads the library holds these bytes until the process
// exits.  Its contents persist between calls; the transform overwrites every byte it reads back,
// so nothing needs clearing.
static __device__ __align__(256) unsigned char g_noalloc_scratch[MQ_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch, looked up once per device.  In host code the array's name
// only stands for the symbol; its device address must come from cudaGetSymbolAddress.
static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[64];

static int noalloc_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return mq_cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return mq_fail(MQ_ERR_ARG, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return mq_cuda_fail(e, "cudaGetSymbolAddress(staging buffer)");
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return MQ_OK;
}

static PassArgs noalloc_pass(const ntt_plan *p, size_t batch) {
    PassArgs a;
    memset(&a, 0, sizeof a);
    a.tw = p->tw_fwd;
    memcpy(a.q, p->q, sizeof a.q);
    memcpy(a.sc, p->sc, sizeof a.sc);
    memcpy(a.scp, p->scp, sizeof a.scp);
    memcpy(a.ws, p->ws, sizeof a.ws);
    memcpy(a.wsp, p->wsp, sizeof a.wsp);
    a.batch = batch;
    a.logN = (int)p->log2n;
    a.L1 = p->L1;
    return a;
}

extern "C" int ntt_forward_noalloc(const ntt_plan *p, void *d, size_t batch, size_t stride, void *stream) {
    MQ_TRACE("ntt_forward_noalloc");
    if (!p) return mq_fail(MQ_ERR_ARG, "plan is NULL");
    if (p->flags & MQ_CHECK_INPUTS)
        return mq_fail(MQ_ERR_ARG, "ntt_forward_noalloc does not run the input check: use a plan without MQ_CHECK_INPUTS");
    if (batch == 0) return MQ_OK;
    int rc = mq_check_ptr(d, p->width, "d_data");
    if (rc) return rc;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return mq_cuda_fail(e, "cudaGetDevice");
    if (dev != p->device) return mq_fail(MQ_ERR_ARG, "the plan belongs to device %d, device %d is current", p->device, dev);
    const size_t N = (size_t)1 << p->log2n;
    if (batch == 1) stride = N;
    if (stride < N) return mq_fail(MQ_ERR_SIZE, "stride %zu is shorter than N = %zu", stride, N);
    // the bound of ntt_forward: batch * stride residues of up to 32 bytes stay addressable
    if (batch > (SIZE_MAX / 32) / stride) return mq_fail(MQ_ERR_ARG, "batch * stride overflows");
    cudaStream_t s = (cudaStream_t)stream;
    const bool natural = !(p->flags & MQ_ORDER_BITREV);
    const int logN = (int)p->log2n, L1 = p->L1, L2 = logN - L1;

    if (L1 == 0) {  // one pass, in place: no staging
        PassArgs a = noalloc_pass(p, batch);
        a.in = a.out = d;
        a.in_stride = a.out_stride = stride;
        a.in_layout = LAYOUT_ROW;
        a.out_layout = natural ? LAYOUT_NAT : LAYOUT_ROW;
        a.final = 1;
        e = launch_ntt_pass(p->width, logN, false, a, s);
        return e == cudaSuccess ? MQ_OK : mq_cuda_fail(e, "NTT pass launch");
    }

    void *scr = nullptr;
    if (natural) {
        // batch * N <= batch * stride < SIZE_MAX / 32 (checked above), so this product cannot wrap
        const size_t need = batch * N * 8u * (size_t)p->width;
        if (need > (size_t)MQ_NOALLOC_SCRATCH_BYTES)
            return mq_fail(MQ_ERR_SIZE,
                           "ntt_forward_noalloc: %zu polynomials of N = %zu need %zu staging bytes, the static "
                           "buffer holds %zu; split the batch",
                           batch, N, need, (size_t)MQ_NOALLOC_SCRATCH_BYTES);
        rc = noalloc_scratch(&scr);
        if (rc) return rc;
    }
    PassArgs col = noalloc_pass(p, batch), row = noalloc_pass(p, batch);
    col.col = 1;
    col.in_layout = col.out_layout = LAYOUT_COL;
    col.in = d;
    col.in_stride = stride;
    col.out = natural ? scr : d;
    col.out_stride = natural ? N : stride;
    row.in = col.out;
    row.in_stride = col.out_stride;
    row.out = d;
    row.out_stride = stride;
    row.perm = natural;
    row.in_layout = LAYOUT_ROW;
    row.out_layout = natural ? LAYOUT_NAT : LAYOUT_ROW;
    row.final = 1;
    e = launch_ntt_pass(p->width, L1, false, col, s);
    if (e == cudaSuccess) e = launch_ntt_pass(p->width, L2, false, row, s);
    return e == cudaSuccess ? MQ_OK : mq_cuda_fail(e, "NTT pass launch");
}

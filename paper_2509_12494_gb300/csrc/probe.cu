// probe.cu -- microbenchmarks that measure the roofline denominators of this library's kernels:
// the issue rate of the 32-bit integer multiply-add instructions the residue layer is built from,
// across all SMs.  (HBM bandwidth is measured separately by a plain device copy.)
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mqntt_probe.h"

int mq_cuda_fail(cudaError_t e, const char *where);
int mq_fail(int code, const char *fmt, ...);

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int CHAINS = 8;   // independent dependency chains per thread
constexpr int UNROLL = 16;  // multiply-adds per chain per loop iteration

__global__ void __launch_bounds__(PROBE_THREADS) probe_kernel(uint32_t *out, int iters, uint32_t b, int kind) {
    uint32_t a[CHAINS], c[CHAINS];
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) {
        a[i] = threadIdx.x * 2654435761u + i;
        c[i] = blockIdx.x + i;
    }
    if (kind == MQ_PROBE_MAD_LO) {
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < UNROLL; ++k) {
#pragma unroll
                for (int i = 0; i < CHAINS; ++i) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[i]) : "r"(b), "r"(c[i]));
            }
        }
    } else if (kind == MQ_PROBE_MAD_HI) {
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < UNROLL; ++k) {
#pragma unroll
                for (int i = 0; i < CHAINS; ++i) asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(a[i]) : "r"(b), "r"(c[i]));
            }
        }
    } else if (kind == MQ_PROBE_MAD_WIDE) {  // 32 x 32 -> 64 multiply-adds, 64-bit accumulators
        unsigned long long w[CHAINS];
#pragma unroll
        for (int i = 0; i < CHAINS; ++i) w[i] = ((unsigned long long)c[i] << 32) | a[i];
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < UNROLL; ++k) {
#pragma unroll
                for (int i = 0; i < CHAINS; ++i) asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(w[i]) : "r"(b), "r"(c[i]));
            }
        }
#pragma unroll
        for (int i = 0; i < CHAINS; ++i) a[i] = (uint32_t)(w[i] ^ (w[i] >> 32));
    } else if (kind == MQ_PROBE_MAD_HI_CC) {  // high halves that write the carry flag
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < UNROLL; ++k) {
#pragma unroll
                for (int i = 0; i < CHAINS; ++i) asm volatile("mad.hi.cc.u32 %0, %0, %1, %2;" : "+r"(a[i]) : "r"(b), "r"(c[i]));
            }
        }
    } else if (kind == MQ_PROBE_MAD_LO_HI_END) {  // mad.lo.cc then madc.hi without carry-out
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < UNROLL / 2; ++k) {
#pragma unroll
                for (int i = 0; i < CHAINS; i += 2)
                    asm volatile(
                        "mad.lo.cc.u32  %0, %2, %3, %0;\n\t"
                        "madc.hi.u32    %1, %2, %3, %1;"
                        : "+r"(a[i]), "+r"(a[i + 1])
                        : "r"(c[i]), "r"(b));
            }
        }
    } else {  // carry-chained pairs, the shape of the schoolbook product rows
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < UNROLL / 2; ++k) {
#pragma unroll
                for (int i = 0; i < CHAINS; i += 2)
                    asm volatile(
                        "mad.lo.cc.u32  %0, %2, %4, %0;\n\t"
                        "madc.hi.cc.u32 %1, %2, %4, %1;\n\t"
                        "madc.lo.cc.u32 %0, %3, %4, %0;\n\t"
                        "madc.hi.u32    %1, %3, %4, %1;"
                        : "+r"(a[i]), "+r"(a[i + 1])
                        : "r"(c[i]), "r"(c[i + 1]), "r"(b));
            }
        }
    }
    uint32_t x = 0;
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) x ^= a[i];
    out[blockIdx.x * PROBE_THREADS + threadIdx.x] = x;
}

}  // namespace

extern "C" int mq_probe_imad_rate(int kind, int iters, double *inst_per_s, double *ms, void *stream) {
    if (kind < MQ_PROBE_MAD_LO || kind > MQ_PROBE_MAD_LO_HI_END) return mq_fail(-1, "unknown probe kind %d", kind);
    if (iters <= 0 || !inst_per_s) return mq_fail(-1, "iters must be positive and inst_per_s non-NULL");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, probe_kernel, PROBE_THREADS, 0);
    if (per_sm < 1) per_sm = 1;
    const int blocks = sms * per_sm;
    uint32_t *out = nullptr;
    cudaError_t e = cudaMalloc(&out, (size_t)blocks * PROBE_THREADS * sizeof(uint32_t));
    if (e != cudaSuccess) return mq_cuda_fail(e, "probe buffer");
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    probe_kernel<<<blocks, PROBE_THREADS, 0, s>>>(out, 1, 3u, kind);  // warm-up
    cudaEventRecord(t0, s);
    probe_kernel<<<blocks, PROBE_THREADS, 0, s>>>(out, iters, 0x9E3779B9u, kind);
    cudaEventRecord(t1, s);
    e = cudaEventSynchronize(t1);
    float dt = 0;
    cudaEventElapsedTime(&dt, t0, t1);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFree(out);
    if (e != cudaSuccess) return mq_cuda_fail(e, "probe kernel");
    const double inst = (double)blocks * PROBE_THREADS * (double)iters * UNROLL * CHAINS;
    *inst_per_s = inst / (dt * 1e-3);
    if (ms) *ms = dt;
    return 0;
}

/*
 * mqntt_probe.h -- measurement probes for the roofline of the modular kernels.
 *
 * The paper locates the cost of 128-bit modular arithmetic in word multiplies and carries
 * (Sec. 4: the widening multiply and add-with-carry are the missing AVX-512 pieces; Sec. 5.3:
 * widening multiply matters most).  On the GPU these are 32-bit multiply-add instructions
 * (mad.lo / mad.hi, with carry-chained variants), so the compute roof of the transforms is the
 * device's issue rate of those instructions.  This probe measures it; it is not a published figure.
 */
#ifndef MQNTT_PROBE_H
#define MQNTT_PROBE_H

#ifdef __cplusplus
extern "C" {
#endif

#define MQ_PROBE_MAD_LO 0 /* independent mad.lo.u32 chains */
#define MQ_PROBE_MAD_HI 1 /* independent mad.hi.u32 chains */
#define MQ_PROBE_MAD_CC 2 /* carry-chained mad.lo.cc / madc.hi.cc pairs */
#define MQ_PROBE_MAD_WIDE 3 /* independent mad.wide.u32 chains (32 x 32 + 64 -> 64) */
#define MQ_PROBE_MAD_HI_CC 4 /* independent mad.hi.cc.u32 chains (carry flag written, unused) */
#define MQ_PROBE_MAD_LO_HI_END 5 /* pairs mad.lo.cc + madc.hi (no carry-out), a row's last limb */

/*
 * Run `iters` loop iterations of the chosen multiply-add pattern on every SM (one full wave of
 * resident CTAs), timed with CUDA events on `stream` (a cudaStream_t; synchronises it).
 * Writes the aggregate rate in thread-instructions per second to *inst_per_s and the kernel
 * time to *ms (may be NULL).  Returns 0, or a negative MQ_ERR_* code (see mqntt.h).
 */
int mq_probe_imad_rate(int kind, int iters, double *inst_per_s, double *ms, void *stream);

/*
 * The two forms of the double-word product of Sec. 2.2 for the general 124-bit modular product
 * (Barrett, Sec. 2.1, Eq. 4): the schoolbook product (Eq. 8: all sixteen 32 x 32 limb products,
 * the form the library's kernels use) and the Karatsuba product (Eq. 9: three 64 x 64 products of
 * the halves and their sums, with 65-bit middle terms).  The paper found schoolbook 1.1x faster
 * on one CPU core; these probes measure the same choice on the GPU.
 */
#define MQ_MUL_SCHOOLBOOK 0
#define MQ_MUL_KARATSUBA 1

/*
 * c[i] = a[i] * b[i] mod q for i < n with the chosen product form; 128-bit residues ({lo, hi}
 * 64-bit words, canonical, < q), q odd < 2^124.  d_c, d_a, d_b: device pointers, 16-byte aligned
 * (d_c may equal d_a or d_b).  Asynchronous on `stream`.  Errors: MQ_ERR_ARG, MQ_ERR_ALIGN,
 * MQ_ERR_MODULUS, MQ_ERR_CUDA.
 */
int mq_probe_mulmod(int variant, void *d_c, const void *d_a, const void *d_b, size_t n, const uint64_t q[2],
                    void *stream);

/*
 * Throughput of the general product with the chosen form on register-resident operands below
 * 2^(bitlen(q) - 1): one full wave of CTAs, each thread `iters` steps of four independent chains
 * x <- x * y mod q, timed with CUDA events on `stream` (synchronises it).  Writes products per
 * second to *mulmod_per_s and the kernel time to *ms (may be NULL).  Errors: as mq_probe_mulmod.
 */
int mq_probe_mulmod_rate(int variant, int iters, const uint64_t q[2], double *mulmod_per_s, double *ms, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MQNTT_PROBE_H */

/*
 * mqntt.h -- multi-word modular NTT and BLAS on one GB300 (sm_103a): the C ABI.
 *
 * The library computes the two data-parallel kernels of "Towards Closing the Performance Gap for
 * Cryptographic Kernels Between CPUs and Specialized Hardware" (Zhang, Fu, Franchetti, MICRO '25)
 * over 64-bit and 128-bit residues:
 *   - modular BLAS (Sec. 2.3, point-wise polynomial operations): vector add, vector subtract,
 *     point-wise vector multiply and axpy y = a x + y, all mod q;
 *   - the number theoretic transform (Sec. 2.3, Eq. 11) and its inverse, negacyclic (x^N + 1) by
 *     default or cyclic (x^N - 1).
 * Every result is the exact canonical residue in [0, q): the arithmetic is integer only.
 *
 * Conventions shared by every entry point:
 *   - Every function returns an int status: MQ_OK (0) or a negative MQ_ERR_* code.  A thread-local
 *     message describing the last failure is available from mq_last_error().
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Compute calls
 *     are asynchronous on that stream; errors of earlier asynchronous work surface at a later call.
 *   - Residues: width MQ_W64 stores one residue per 64-bit word (q < 2^60); width MQ_W128 stores one
 *     residue per two 64-bit words, low word first (the memory image of an unsigned 128-bit
 *     integer; q < 2^124, the 124-bit bound of Sec. 2.1 that keeps Barrett's constant in range).
 *     Widths MQ_W192 and MQ_W256 store three and four words (q < 2^188, q < 2^252), the larger
 *     bit-widths of Sec. 7; they take the transforms (N <= 2^20) and the BLAS ops, not the fused
 *     product, the batched form or the server.  Moduli, roots and scalars are passed as
 *     max(width, 2) 64-bit words, low first; for MQ_W64 the high word must be 0.
 *   - q must be odd and at least 3.  Primality is the caller's responsibility for the NTT (the
 *     plan checks the root's order, which needs a field to mean anything); the BLAS ops are exact
 *     for any odd q.
 *   - Inputs must be canonical (< q); non-canonical inputs give unspecified (but memory-safe)
 *     results.
 *   - Device pointers are caller-owned device memory (for example torch tensors) and must be
 *     aligned to the residue size (8, 16, 8 and 32 bytes for widths 1 to 4); MQ_ERR_ALIGN
 *     otherwise.
 */
#ifndef MQNTT_H
#define MQNTT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define MQ_OK 0
#define MQ_ERR_ARG (-1)      /* null pointer, bad width, bad flag, size overflow */
#define MQ_ERR_MODULUS (-2)  /* q even, q < 3, too wide for the width, or not 1 mod (2)N */
#define MQ_ERR_ROOT (-3)     /* root not < q or not of the exact order the transform needs */
#define MQ_ERR_SIZE (-4)     /* log2 N outside [1, 24], or a stride shorter than N */
#define MQ_ERR_ALIGN (-5)    /* a device pointer not aligned to the residue size */
#define MQ_ERR_OOM (-6)      /* device memory allocation failed */
#define MQ_ERR_CUDA (-7)     /* a CUDA runtime call failed (message has the CUDA error) */
#define MQ_ERR_TIMEOUT (-8)  /* a bounded device-side wait gave up */
#define MQ_ERR_RANGE (-9)    /* an input residue was not canonical (checked modes only) */
#define MQ_ERR_STATE (-10)   /* object in the wrong state for the call */
#define MQ_ERR_CANCELLED (-11) /* a served request was cancelled before it ran (mqntt_serve.h) */

/* residue widths */
#define MQ_W64 1  /* uint64_t residues, q < 2^60 */
#define MQ_W128 2 /* {lo, hi} uint64_t pairs, q < 2^124 */
#define MQ_W192 3 /* three uint64_t words, low first, q < 2^188 (transforms up to N = 2^20) */
#define MQ_W256 4 /* four uint64_t words, low first, q < 2^252 (transforms up to N = 2^20) */

/* plan flags */
#define MQ_NEGACYCLIC 0u    /* modulus x^N + 1; root = psi, a primitive 2N-th root of unity */
#define MQ_CYCLIC 1u        /* modulus x^N - 1 (Eq. 11); root = w, a primitive N-th root of unity */
#define MQ_ORDER_NATURAL 0u /* transformed side in natural order: position k holds yhat_k */
#define MQ_ORDER_BITREV 2u  /* transformed side in bit-reversed order: position i holds yhat_brv(i) */

/*
 * Input checking (Sec. 2.1: the modular operations are defined for canonical operands, 0 <= a, b < q).
 * As a plan flag, every ntt_forward / ntt_inverse / ntt_polymul call on the plan first checks that
 * the residues it will read (the first N of each polynomial; a and b for the product) are below q.
 * OR-ed into the `width` argument of a BLAS call (for example MQ_W128 | MQ_CHECK_INPUTS), the call
 * checks its inputs (a and b; axpy: x and y).  A checked call runs a read-only range-check kernel on
 * its stream, reads the result back (it synchronises the stream, so it cannot be captured in a
 * graph) and returns MQ_ERR_RANGE, naming the operand, without running the operation when a residue
 * is >= q: the outputs are then untouched.  ntt_forward_noalloc refuses checked plans (the check
 * needs a result word of device memory).  Batched jobs: see mqntt_batch.h.  Unchecked calls are
 * unchanged: non-canonical inputs give unspecified (but memory-safe) results.
 */
#define MQ_CHECK_INPUTS 0x100u

typedef struct ntt_plan ntt_plan;

/*
 * Create a transform plan for N = 2^log2n residues mod q (Sec. 2.3, Eq. 11).
 *   negacyclic (default): yhat_k = sum_j x_j psi^((2k+1) j) mod q, q = 1 mod 2N, root = psi with
 *                         psi^N = -1 (order exactly 2N);
 *   cyclic:               y_k = sum_j x_j w^(jk) mod q, q = 1 mod N, root = w with w^(N/2) = -1.
 * The plan validates q and the root's exact order, then builds device-resident twiddle tables
 * (N entries per direction, each a power of the root and its Shoup companion) on `stream`; the
 * call returns after they are built.  `q` and `root` are two words each, low first.
 * log2n in [1, 24].  flags: MQ_CYCLIC, MQ_ORDER_BITREV and MQ_CHECK_INPUTS, OR-ed.  The plan
 * owns its device memory until ntt_plan_destroy.
 * Errors: MQ_ERR_ARG, MQ_ERR_MODULUS, MQ_ERR_ROOT, MQ_ERR_SIZE, MQ_ERR_OOM, MQ_ERR_CUDA.
 */
int ntt_plan_create(ntt_plan **out, unsigned log2n, const uint64_t q[2], const uint64_t root[2], int width,
                    unsigned flags, void *stream);

/* Free a plan (synchronises with the device first).  NULL is accepted. */
int ntt_plan_destroy(ntt_plan *plan);

/*
 * In-place forward transform of `batch` polynomials; polynomial b starts at residue b * stride
 * of d_data (stride >= N when batch > 1).  Input in natural coefficient order; output in the
 * plan's order.  batch == 0 is a no-op.  Natural-order transforms with N > 2^12 stage through a
 * temporary device buffer of batch * N residues taken from the library's stream-ordered pool.
 * Errors: MQ_ERR_ARG, MQ_ERR_ALIGN, MQ_ERR_SIZE, MQ_ERR_OOM, MQ_ERR_CUDA; MQ_ERR_RANGE (checked plans).
 */
int ntt_forward(const ntt_plan *plan, void *d_data, size_t batch, size_t stride, void *stream);

/*
 * In-place inverse transform (with the factor N^-1, so that ntt_inverse(ntt_forward(x)) = x).
 * Input in the plan's order, output in natural coefficient order.  Same arguments and errors as
 * ntt_forward.
 */
int ntt_inverse(const ntt_plan *plan, void *d_data, size_t batch, size_t stride, void *stream);

/*
 * Polynomial product through the NTT (Sec. 2.3, polynomial multiplication using NTT): for each of
 * `batch` polynomials, c = a * b in Z_q[X]/(X^N + 1) -- the negacyclic product, the ring of FHE --
 * with the plan's N and q (a plan created with MQ_CYCLIC gives the cyclic product, mod X^N - 1).
 * Computes the inverse transform of the pointwise product of the two forward transforms, with the
 * pointwise product fused into the pass that holds the last forward and the first inverse stages
 * (for N <= 2^12 the whole product is one kernel).  The plan's order flag does not matter.
 * d_c, d_a, d_b: device buffers of `batch` polynomials `stride` residues apart (stride >= N;
 * ignored if batch = 1), coefficients canonical (< q) in natural order, 8 * width-byte aligned;
 * the result is canonical, in natural order.  d_c may be d_a or d_b (in place); other overlaps
 * are undefined.  a and b are not modified unless c is one of them.  For N > 2^12 the call takes
 * batch * N residues of stream-ordered scratch from the library's pool.  batch == 0 is a no-op.
 * Errors: MQ_ERR_ARG, MQ_ERR_ALIGN, MQ_ERR_SIZE, MQ_ERR_OOM, MQ_ERR_CUDA; MQ_ERR_RANGE (checked plans).
 */
int ntt_polymul(const ntt_plan *plan, void *d_c, const void *d_a, const void *d_b, size_t batch, size_t stride,
                void *stream);

/*
 * ntt_forward without any device allocation (the paper has no counterpart: this is a deployment
 * variant).  For callers that cannot allocate device memory while running -- a service that
 * reserves its memory budget at start-up, code sharing the GPU with a framework whose allocator
 * owns the free memory, code recorded into a graph that must not contain allocation nodes.
 * Same arguments and results as ntt_forward.  Natural-order transforms with N > 2^12 stage through
 * a static device buffer of MQ_NOALLOC_SCRATCH_BYTES that the library holds on every device that
 * loads it, until the process exits; a call needing more (batch * N * 8 * width bytes) fails with
 * MQ_ERR_SIZE -- split the batch.  Other transforms need no staging and take any batch.
 * The buffer is shared by all calls: calls that overlap on the GPU (different streams, or
 * different host threads without ordering) race on it and give wrong results.  The first call on
 * each device looks up the buffer's device address (cudaGetSymbolAddress, which may load the
 * library's device code); make that first call before any stream capture.
 * Errors: those of ntt_forward, except MQ_ERR_OOM; MQ_ERR_SIZE for an oversized batch;
 * MQ_ERR_ARG if the plan belongs to another device than the current one or was created with
 * MQ_CHECK_INPUTS.
 */
#define MQ_NOALLOC_SCRATCH_BYTES (16u << 20) /* 16 MiB */
int ntt_forward_noalloc(const ntt_plan *plan, void *d_data, size_t batch, size_t stride, void *stream);

/* Plan properties (for callers that size buffers from a plan). */
int ntt_plan_info(const ntt_plan *plan, unsigned *log2n, int *width, unsigned *flags);

/*
 * Element-wise modular BLAS over n residues (Sec. 2.3; modular ring operations of Sec. 2.1, Eq. 1).
 *   mod_vadd: c_i = a_i + b_i mod q      mod_vsub: c_i = a_i - b_i mod q
 *   mod_vmul: c_i = a_i * b_i mod q      mod_axpy: y_i = a * x_i + y_i mod q (scalar a < q)
 * Any n (0 is a no-op).  The output may alias any input.  `width` may carry MQ_CHECK_INPUTS (see
 * above).  Errors: MQ_ERR_ARG, MQ_ERR_MODULUS, MQ_ERR_ALIGN, MQ_ERR_CUDA; MQ_ERR_RANGE (scalar a not
 * below q, or a checked input residue not below q).
 */
int mod_vadd(void *d_c, const void *d_a, const void *d_b, size_t n, const uint64_t q[2], int width, void *stream);
int mod_vsub(void *d_c, const void *d_a, const void *d_b, size_t n, const uint64_t q[2], int width, void *stream);
int mod_vmul(void *d_c, const void *d_a, const void *d_b, size_t n, const uint64_t q[2], int width, void *stream);
int mod_axpy(void *d_y, const uint64_t a[2], const void *d_x, size_t n, const uint64_t q[2], int width,
             void *stream);

/* Message for the last failing call on this thread ("" if none). */
const char *mq_last_error(void);

/* Library version string. */
const char *mq_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MQNTT_H */

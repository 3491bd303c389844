// api.cu -- the C ABI of include/mqntt.h: argument checks, plans, pass scheduling, BLAS dispatch.
//
// Host-side scalar precomputation (Barrett constants, Shoup companions of scalars, the inverse
// root, N^-1) uses unsigned __int128 and binary long division; the per-residue work -- twiddle
// tables, transforms, BLAS -- runs in the kernels of ntt.cu and blas.cu.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "../../include/mqntt.h"
#include "check.h"
#include "common.cuh"
#include "hostmath.h"
#include "plan.h"
#include "trace.h"
#include "widehost.h"

using namespace mq;

// ------------------------------------------------------------------------------------------------
// errors
// ------------------------------------------------------------------------------------------------

static thread_local char g_err[512];

int mq_fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int mq_cuda_fail(cudaError_t e, const char *where) {
    return mq_fail(MQ_ERR_CUDA, "%s: %s (%s)", where, cudaGetErrorString(e), cudaGetErrorName(e));
}

extern "C" const char *mq_last_error(void) { return g_err; }
extern "C" const char *mq_version(void) { return "mqntt 0.1 (sm_103a)"; }

// ------------------------------------------------------------------------------------------------
// modulus checks shared by the BLAS and the plans
// ------------------------------------------------------------------------------------------------

int mq_check_modulus(const uint64_t q[2], int width, hm::u128 *qv) {
    if (!q) return mq_fail(MQ_ERR_ARG, "q is NULL");
    if (width != MQ_W64 && width != MQ_W128) return mq_fail(MQ_ERR_ARG, "width must be MQ_W64 or MQ_W128 here, got %d", width);
    hm::u128 v = hm::from_words(q);
    if (v < 3 || (v & 1) == 0) return mq_fail(MQ_ERR_MODULUS, "q must be odd and >= 3");
    if (width == MQ_W64 && (q[1] != 0 || hm::bitlen(v) > 60)) return mq_fail(MQ_ERR_MODULUS, "MQ_W64 needs q < 2^60");
    if (width == MQ_W128 && hm::bitlen(v) > 124) return mq_fail(MQ_ERR_MODULUS, "MQ_W128 needs q < 2^124");
    *qv = v;
    return MQ_OK;
}

// alignment a residue array needs: its vector loads (one word for 192-bit residues)
static unsigned align_of(int width) { return width == 3 ? 8u : 8u * (unsigned)width; }

int mq_check_ptr(const void *p, int width, const char *name) {
    if (!p) return mq_fail(MQ_ERR_ARG, "%s is NULL", name);
    if (((uintptr_t)p) % align_of(width)) return mq_fail(MQ_ERR_ALIGN, "%s is not %u-byte aligned", name, align_of(width));
    return MQ_OK;
}
static int check_ptr(const void *p, int width, const char *name) { return mq_check_ptr(p, width, name); }

// residues of three and four words: q odd, 3 <= q < 2^(64 width - 4), so that 16q fits the word
static int check_modulus_wide(const uint64_t *q, int width, hw::U *qv) {
    if (!q) return mq_fail(MQ_ERR_ARG, "q is NULL");
    hw::U v = hw::from_words(q, width);
    if (hw::cmp(v, hw::from_u64(3)) < 0 || (v.w[0] & 1) == 0) return mq_fail(MQ_ERR_MODULUS, "q must be odd and >= 3");
    if (hw::bitlen(v) > 64 * width - 4)
        return mq_fail(MQ_ERR_MODULUS, "width %d needs q < 2^%d", width, 64 * width - 4);
    *qv = v;
    return MQ_OK;
}

// ------------------------------------------------------------------------------------------------
// stream-ordered scratch pool (one per device, created on first use, memory kept cached)
// ------------------------------------------------------------------------------------------------

static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64];
static bool g_pool_ok[64];

int mq_pool_alloc(void **p, size_t bytes, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return mq_cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return mq_fail(MQ_ERR_ARG, "device index %d out of range", dev);
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (!g_pool_ok[dev]) {
            cudaMemPoolProps props;
            memset(&props, 0, sizeof props);
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            e = cudaMemPoolCreate(&g_pool[dev], &props);
            if (e != cudaSuccess) return mq_cuda_fail(e, "cudaMemPoolCreate");
            uint64_t keep = ~0ull;
            cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep);
            g_pool_ok[dev] = true;
        }
    }
    e = cudaMallocFromPoolAsync(p, bytes, g_pool[dev], s);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return mq_fail(MQ_ERR_OOM, "scratch allocation of %zu bytes failed", bytes);
    }
    if (e != cudaSuccess) return mq_cuda_fail(e, "cudaMallocFromPoolAsync");
    return MQ_OK;
}

int mq_pool_free(void *p, cudaStream_t s) {
    cudaError_t e = cudaFreeAsync(p, s);
    return e == cudaSuccess ? MQ_OK : mq_cuda_fail(e, "cudaFreeAsync");
}

// bytes the current device's pool holds without having handed them out (0 before its first use):
// memory a new allocation can take besides what the device reports free
size_t mq_pool_idle_bytes() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool_ok[dev]) return 0;
    uint64_t reserved = 0, used = 0;
    if (cudaMemPoolGetAttribute(g_pool[dev], cudaMemPoolAttrReservedMemCurrent, &reserved) != cudaSuccess ||
        cudaMemPoolGetAttribute(g_pool[dev], cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess)
        return 0;
    return reserved > used ? (size_t)(reserved - used) : 0;
}

// ------------------------------------------------------------------------------------------------
// plans
// ------------------------------------------------------------------------------------------------

static int split_of(unsigned log2n) { return log2n <= 12 ? 0 : (int)(log2n / 2); }

// wide residues: tiles of up to 2^10 (four residues per thread), so N <= 2^20
static int split_of_wide(unsigned log2n) { return log2n <= 10 ? 0 : (int)(log2n / 2); }

static int plan_create_wide(ntt_plan **out, unsigned log2n, const uint64_t *q, const uint64_t *root, int width,
                            unsigned flags, cudaStream_t s) {
    if (log2n > 20) return mq_fail(MQ_ERR_SIZE, "residues of %d words need log2n <= 20, got %u", width, log2n);
    hw::U Q;
    int rc = check_modulus_wide(q, width, &Q);
    if (rc) return rc;
    const int cyclic = (flags & MQ_CYCLIC) != 0;
    const unsigned lord = log2n + (cyclic ? 0 : 1);  // log2 of the root's order
    const hw::U Qm1 = hw::sub(Q, hw::from_u64(1));
    if (Qm1.w[0] & ((1ull << lord) - 1)) return mq_fail(MQ_ERR_MODULUS, "q - 1 is not divisible by %s", cyclic ? "N" : "2N");
    const hw::U r = hw::from_words(root, width);
    if (hw::bitlen(r) == 0 || hw::cmp(r, Q) >= 0) return mq_fail(MQ_ERR_ROOT, "root must be in [1, q)");
    if (hw::cmp(hw::powmod(r, 1ull << (lord - 1), Q), Qm1) != 0)
        return mq_fail(MQ_ERR_ROOT, "root is not a primitive %s root of unity", cyclic ? "N-th" : "2N-th");

    ntt_plan *p = new ntt_plan();
    memset(p, 0, sizeof *p);
    cudaGetDevice(&p->device);
    p->log2n = log2n;
    p->width = width;
    p->flags = flags;
    p->L = hw::bitlen(Q);
    hw::to_words(Q, p->q, width);
    hw::to_words(hw::barrett_mu(Q, p->L), p->mu, width);
    hw::to_words(r, p->root, width);
    const hw::U rinv = hw::powmod(r, (1ull << lord) - 1, Q);
    hw::to_words(rinv, p->root_inv, width);
    const int B = 64 * width;
    const hw::U ninv = hw::sub(Q, hw::shr(Qm1, (int)log2n));  // q - (q - 1) / N: N times it is 1 mod q
    const hw::U t1 = cyclic ? hw::from_u64(1) : hw::powmod(rinv, 1ull << (log2n - 1), Q);  // inverse-table entry 1
    const hw::U ws = hw::mulmod(t1, ninv, Q);
    hw::to_words(ninv, p->sc, width);
    hw::to_words(hw::shoup(ninv, Q, B), p->scp, width);
    hw::to_words(ws, p->ws, width);
    hw::to_words(hw::shoup(ws, Q, B), p->wsp, width);
    p->L1 = split_of_wide(log2n);

    size_t bytes = ((size_t)1 << log2n) * 16u * (size_t)width;
    cudaError_t e = cudaMalloc(&p->tw_fwd, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&p->tw_inv, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ntt_plan_destroy(p);
        return mq_fail(MQ_ERR_OOM, "twiddle tables (%zu bytes) do not fit", 2 * bytes);
    }
    e = launch_twiddle_build(width, (int)log2n, cyclic, p->q, p->root, p->root_inv, p->mu, p->L, p->tw_fwd, p->tw_inv, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        ntt_plan_destroy(p);
        return mq_cuda_fail(e, "twiddle build");
    }
    *out = p;
    return MQ_OK;
}

extern "C" int ntt_plan_create(ntt_plan **out, unsigned log2n, const uint64_t q[2], const uint64_t root[2], int width,
                               unsigned flags, void *stream) {
    MQ_TRACE("ntt_plan_create");
    if (!out) return mq_fail(MQ_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!root) return mq_fail(MQ_ERR_ARG, "root is NULL");
    if (flags & ~(MQ_CYCLIC | MQ_ORDER_BITREV | MQ_CHECK_INPUTS)) return mq_fail(MQ_ERR_ARG, "unknown flag bits 0x%x", flags);
    if (log2n < 1 || log2n > 24) return mq_fail(MQ_ERR_SIZE, "log2n must be in [1, 24], got %u", log2n);
    if (width == MQ_W192 || width == MQ_W256)
        return plan_create_wide(out, log2n, q, root, width, flags, (cudaStream_t)stream);
    hm::u128 Q;
    int rc = mq_check_modulus(q, width, &Q);
    if (rc) return rc;
    const int cyclic = (flags & MQ_CYCLIC) != 0;
    const hm::u128 N = (hm::u128)1 << log2n;
    const hm::u128 order = cyclic ? N : 2 * N;
    if ((Q - 1) % order != 0) return mq_fail(MQ_ERR_MODULUS, "q - 1 is not divisible by %s", cyclic ? "N" : "2N");
    hm::u128 r = hm::from_words(root);
    if (r == 0 || r >= Q) return mq_fail(MQ_ERR_ROOT, "root must be in [1, q)");
    // exact order: psi^N = -1 (order 2N) or w^(N/2) = -1 (order N); orders are powers of two
    if (hm::powmod(r, order / 2, Q) != Q - 1)
        return mq_fail(MQ_ERR_ROOT, "root is not a primitive %s root of unity", cyclic ? "N-th" : "2N-th");

    ntt_plan *p = new ntt_plan();
    memset(p, 0, sizeof *p);
    cudaGetDevice(&p->device);
    p->log2n = log2n;
    p->width = width;
    p->flags = flags;
    p->L = hm::bitlen(Q);
    hm::to_words(Q, p->q);
    hm::to_words(hm::barrett_mu(Q, p->L), p->mu);
    hm::to_words(r, p->root);
    hm::u128 rinv = hm::powmod(r, order - 1, Q);
    hm::to_words(rinv, p->root_inv);
    const int B = width == MQ_W64 ? 64 : 128;
    hm::u128 ninv = Q - (Q - 1) / N;  // N * (q-1)/N = -1 mod q
    hm::u128 t1 = cyclic ? 1 : hm::powmod(rinv, N / 2, Q);  // inverse-table entry 1
    hm::u128 ws = hm::mulmod(t1, ninv, Q);
    hm::to_words(ninv, p->sc);
    hm::to_words(hm::shoup(ninv, Q, B), p->scp);
    hm::to_words(ws, p->ws);
    hm::to_words(hm::shoup(ws, Q, B), p->wsp);
    p->L1 = split_of(log2n);

    size_t bytes = ((size_t)1 << log2n) * 16u * (size_t)width;
    cudaError_t e = cudaMalloc(&p->tw_fwd, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&p->tw_inv, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ntt_plan_destroy(p);
        return mq_fail(MQ_ERR_OOM, "twiddle tables (%zu bytes) do not fit", 2 * bytes);
    }
    cudaStream_t s = (cudaStream_t)stream;
    e = launch_twiddle_build(width, (int)log2n, cyclic, p->q, p->root, p->root_inv, p->mu, p->L, p->tw_fwd, p->tw_inv, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        ntt_plan_destroy(p);
        return mq_cuda_fail(e, "twiddle build");
    }
    *out = p;
    return MQ_OK;
}

extern "C" int ntt_plan_destroy(ntt_plan *p) {
    if (!p) return MQ_OK;
    cudaDeviceSynchronize();
    if (p->tw_fwd) cudaFree(p->tw_fwd);
    if (p->tw_inv) cudaFree(p->tw_inv);
    delete p;
    return MQ_OK;
}

extern "C" int ntt_plan_info(const ntt_plan *p, unsigned *log2n, int *width, unsigned *flags) {
    if (!p) return mq_fail(MQ_ERR_ARG, "plan is NULL");
    if (log2n) *log2n = p->log2n;
    if (width) *width = p->width;
    if (flags) *flags = p->flags;
    return MQ_OK;
}

// Fill the constant part of a pass.
static PassArgs pass_base(const ntt_plan *p, bool inv, size_t batch) {
    PassArgs a;
    memset(&a, 0, sizeof a);
    a.tw = inv ? p->tw_inv : p->tw_fwd;
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

static int run_pass(const ntt_plan *p, bool inv, PassArgs &a, int L, cudaStream_t s) {
    cudaError_t e = launch_ntt_pass(p->width, L, inv, a, s);
    return e == cudaSuccess ? MQ_OK : mq_cuda_fail(e, "NTT pass launch");
}

static int ntt_run(const ntt_plan *p, void *d, size_t batch, size_t stride, void *stream, bool inv) {
    if (!p) return mq_fail(MQ_ERR_ARG, "plan is NULL");
    if (batch == 0) return MQ_OK;
    int rc = check_ptr(d, p->width, "d_data");
    if (rc) return rc;
    const size_t N = (size_t)1 << p->log2n;
    if (batch == 1) stride = N;
    if (stride < N) return mq_fail(MQ_ERR_SIZE, "stride %zu is shorter than N = %zu", stride, N);
    if (batch > (SIZE_MAX / 32) / stride) return mq_fail(MQ_ERR_ARG, "batch * stride overflows");
    cudaStream_t s = (cudaStream_t)stream;
    if (p->flags & MQ_CHECK_INPUTS) {
        const CheckRec r = check_rec(d, batch, N, stride, p->width, p->q, "d_data");
        rc = range_check(&r, 1, s);
        if (rc) return rc;
    }
    const bool natural = !(p->flags & MQ_ORDER_BITREV);
    const int logN = (int)p->log2n, L1 = p->L1, L2 = logN - L1;

    if (L1 == 0) {  // one pass: the whole transform in one tile
        PassArgs a = pass_base(p, inv, batch);
        a.in = a.out = d;
        a.in_stride = a.out_stride = stride;
        a.col = 0;
        a.in_layout = (inv && natural) ? LAYOUT_NAT : LAYOUT_ROW;
        a.out_layout = (!inv && natural) ? LAYOUT_NAT : LAYOUT_ROW;
        a.scale = inv;
        a.final = 1;
        return run_pass(p, inv, a, logN, s);
    }

    void *scr = nullptr;
    if (natural) {
        rc = mq_pool_alloc(&scr, batch * N * 8u * (size_t)p->width, s);
        if (rc) return rc;
    }
    PassArgs col = pass_base(p, inv, batch), row = pass_base(p, inv, batch);
    col.col = 1;
    col.in_layout = col.out_layout = LAYOUT_COL;
    row.col = 0;
    if (!inv) {
        // columns first (stages 0 .. L1-1), then rows
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
        rc = run_pass(p, inv, col, L1, s);
        if (!rc) rc = run_pass(p, inv, row, L2, s);
    } else {
        // rows first (the last forward stages, undone), then columns with the N^-1 scale
        row.in = d;
        row.in_stride = stride;
        row.out = natural ? scr : d;
        row.out_stride = natural ? N : stride;
        row.perm = natural;
        row.in_layout = natural ? LAYOUT_NAT : LAYOUT_ROW;
        row.out_layout = LAYOUT_ROW;
        col.in = row.out;
        col.in_stride = row.out_stride;
        col.out = d;
        col.out_stride = stride;
        col.scale = 1;
        col.final = 1;
        rc = run_pass(p, inv, row, L2, s);
        if (!rc) rc = run_pass(p, inv, col, L1, s);
    }
    if (scr) {
        int rc2 = mq_pool_free(scr, s);
        if (!rc) rc = rc2;
    }
    return rc;
}

extern "C" int ntt_forward(const ntt_plan *p, void *d, size_t batch, size_t stride, void *stream) {
    MQ_TRACE("ntt_forward");
    return ntt_run(p, d, batch, stride, stream, false);
}

extern "C" int ntt_inverse(const ntt_plan *p, void *d, size_t batch, size_t stride, void *stream) {
    MQ_TRACE("ntt_inverse");
    return ntt_run(p, d, batch, stride, stream, true);
}

// c = a * b in Z_q[X]/(X^N + 1) (X^N - 1 for a cyclic plan): forward transforms of a and b in
// bit-reversed order, pointwise product, inverse transform (Sec. 2.3).  The product is fused into
// the pass that holds the last forward and the first inverse stages (polymul.cuh); for N > 2^12 the
// column passes run before (a into c, b into scratch) and after it (inverse, N^-1 folded in).
extern "C" int ntt_polymul(const ntt_plan *p, void *c, const void *a, const void *b, size_t batch, size_t stride,
                           void *stream) {
    MQ_TRACE("ntt_polymul");
    if (!p) return mq_fail(MQ_ERR_ARG, "plan is NULL");
    if (p->width > MQ_W128) return mq_fail(MQ_ERR_ARG, "the fused product takes residues of one or two words");
    if (batch == 0) return MQ_OK;
    int rc;
    if ((rc = check_ptr(c, p->width, "d_c")) || (rc = check_ptr(a, p->width, "d_a")) ||
        (rc = check_ptr(b, p->width, "d_b")))
        return rc;
    const size_t N = (size_t)1 << p->log2n;
    if (batch == 1) stride = N;
    if (stride < N) return mq_fail(MQ_ERR_SIZE, "stride %zu is shorter than N = %zu", stride, N);
    if (batch > (SIZE_MAX / 16) / stride) return mq_fail(MQ_ERR_ARG, "batch * stride overflows");
    cudaStream_t s = (cudaStream_t)stream;
    if (p->flags & MQ_CHECK_INPUTS) {
        const CheckRec r[2] = {check_rec(a, batch, N, stride, p->width, p->q, "d_a"),
                               check_rec(b, batch, N, stride, p->width, p->q, "d_b")};
        rc = range_check(r, 2, s);
        if (rc) return rc;
    }
    const int logN = (int)p->log2n, L1 = p->L1, L2 = logN - L1;
    MulArgs m;
    memcpy(m.q, p->q, sizeof m.q);
    memcpy(m.mu, p->mu, sizeof m.mu);
    m.L = p->L;
    // the fused pass: forward row stages of a (fa) and b (fb), product, inverse row stages (ia)
    PassArgs fa = pass_base(p, false, batch), ia = pass_base(p, true, batch);
    fa.col = ia.col = 0;
    fa.in_layout = fa.out_layout = ia.in_layout = ia.out_layout = LAYOUT_ROW;
    ia.out = c;
    ia.out_stride = stride;
    if (L1 == 0) {  // one pass: the whole product in one kernel
        fa.in = a;
        fa.in_stride = stride;
        PassArgs fb = fa;
        fb.in = b;
        ia.scale = ia.final = 1;
        cudaError_t e = launch_polymul(p->width, logN, fa, fb, ia, m, s);
        return e == cudaSuccess ? MQ_OK : mq_cuda_fail(e, "polynomial product launch");
    }
    void *scr = nullptr;
    rc = mq_pool_alloc(&scr, batch * N * 8u * (size_t)p->width, s);
    if (rc) return rc;
    // forward column passes: b into the scratch first, then a into c (so c may alias a or b)
    PassArgs col = pass_base(p, false, batch);
    col.col = 1;
    col.in_layout = col.out_layout = LAYOUT_COL;
    col.in = b;
    col.in_stride = stride;
    col.out = scr;
    col.out_stride = N;
    rc = run_pass(p, false, col, L1, s);
    if (!rc) {
        col.in = a;
        col.out = c;
        col.out_stride = stride;
        rc = run_pass(p, false, col, L1, s);
    }
    if (!rc) {
        fa.in = c;
        fa.in_stride = stride;
        PassArgs fb = fa;
        fb.in = scr;
        fb.in_stride = N;
        cudaError_t e = launch_polymul(p->width, L2, fa, fb, ia, m, s);
        if (e != cudaSuccess) rc = mq_cuda_fail(e, "polynomial product launch");
    }
    if (!rc) {  // inverse column pass with the N^-1 scale, canonical result
        PassArgs icol = pass_base(p, true, batch);
        icol.col = 1;
        icol.in_layout = icol.out_layout = LAYOUT_COL;
        icol.in = icol.out = c;
        icol.in_stride = icol.out_stride = stride;
        icol.scale = icol.final = 1;
        rc = run_pass(p, true, icol, L1, s);
    }
    int rc2 = mq_pool_free(scr, s);
    return rc ? rc : rc2;
}

// ------------------------------------------------------------------------------------------------
// BLAS
// ------------------------------------------------------------------------------------------------

// The input check of a BLAS call: a and b (axpy: x and y).
static int blas_check(int op, const void *a, const void *b, size_t n, const uint64_t *q, int width, cudaStream_t s) {
    const CheckRec r[2] = {check_rec(a, 1, n, n, width, q, op == OP_AXPY ? "d_x" : "d_a"),
                           check_rec(b, 1, n, n, width, q, op == OP_AXPY ? "d_y" : "d_b")};
    return range_check(r, 2, s);
}

static int blas_wide(int op, void *c, const void *a, const void *b, size_t n, const uint64_t *q, int width,
                     const uint64_t *scalar, bool checked, void *stream) {
    hw::U Q;
    int rc = check_modulus_wide(q, width, &Q);
    if (rc) return rc;
    if (n == 0) return MQ_OK;
    if ((rc = check_ptr(c, width, op == OP_AXPY ? "d_y" : "d_c")) || (rc = check_ptr(a, width, op == OP_AXPY ? "d_x" : "d_a")))
        return rc;
    if (op != OP_AXPY && (rc = check_ptr(b, width, "d_b"))) return rc;
    if (n > SIZE_MAX / 32) return mq_fail(MQ_ERR_ARG, "n overflows");
    BlasWideArgs args;
    memset(&args, 0, sizeof args);
    args.c = c;
    args.a = a;
    args.b = b;
    args.n = n;
    hw::to_words(Q, args.q, width);
    args.L = hw::bitlen(Q);
    hw::to_words(hw::barrett_mu(Q, args.L), args.mu, width);
    if (op == OP_AXPY) {
        if (!scalar) return mq_fail(MQ_ERR_ARG, "scalar a is NULL");
        const hw::U sv = hw::from_words(scalar, width);
        if (hw::cmp(sv, Q) >= 0) return mq_fail(MQ_ERR_RANGE, "scalar a must be < q");
        hw::to_words(sv, args.s, width);
        hw::to_words(hw::shoup(sv, Q, 64 * width), args.sp, width);
    }
    if (checked && (rc = blas_check(op, a, b, n, q, width, (cudaStream_t)stream))) return rc;
    cudaError_t e = launch_blas_wide(width, op, args, (cudaStream_t)stream);
    return e == cudaSuccess ? MQ_OK : mq_cuda_fail(e, "BLAS launch");
}

static int blas(int op, void *c, const void *a, const void *b, size_t n, const uint64_t q[2], int width_arg,
                const uint64_t *scalar, void *stream) {
    const bool checked = ((unsigned)width_arg & MQ_CHECK_INPUTS) != 0;
    const int width = (int)((unsigned)width_arg & ~MQ_CHECK_INPUTS);
    if (width == MQ_W192 || width == MQ_W256) return blas_wide(op, c, a, b, n, q, width, scalar, checked, stream);
    hm::u128 Q;
    int rc = mq_check_modulus(q, width, &Q);
    if (rc) return rc;
    if (n == 0) return MQ_OK;
    if ((rc = check_ptr(c, width, op == OP_AXPY ? "d_y" : "d_c")) || (rc = check_ptr(a, width, op == OP_AXPY ? "d_x" : "d_a")))
        return rc;
    if (op != OP_AXPY && (rc = check_ptr(b, width, "d_b"))) return rc;
    if (n > SIZE_MAX / 16) return mq_fail(MQ_ERR_ARG, "n overflows");
    BlasArgs args;
    memset(&args, 0, sizeof args);
    args.c = c;
    args.a = a;
    args.b = b;
    args.n = n;
    memcpy(args.q, q, sizeof args.q);
    args.L = hm::bitlen(Q);
    hm::to_words(hm::barrett_mu(Q, args.L), args.mu);
    if (op == OP_AXPY) {
        if (!scalar) return mq_fail(MQ_ERR_ARG, "scalar a is NULL");
        hm::u128 s = hm::from_words(scalar);
        if (width == MQ_W64 && scalar[1]) return mq_fail(MQ_ERR_RANGE, "scalar a must be < q");
        if (s >= Q) return mq_fail(MQ_ERR_RANGE, "scalar a must be < q");
        hm::to_words(s, args.s);
        hm::to_words(hm::shoup(s, Q, width == MQ_W64 ? 64 : 128), args.sp);
    }
    if (checked && (rc = blas_check(op, a, b, n, args.q, width, (cudaStream_t)stream))) return rc;
    cudaError_t e = launch_blas(width, op, args, (cudaStream_t)stream);
    return e == cudaSuccess ? MQ_OK : mq_cuda_fail(e, "BLAS launch");
}

extern "C" int mod_vadd(void *c, const void *a, const void *b, size_t n, const uint64_t q[2], int width, void *stream) {
    MQ_TRACE("mod_vadd");
    return blas(OP_VADD, c, a, b, n, q, width, nullptr, stream);
}
extern "C" int mod_vsub(void *c, const void *a, const void *b, size_t n, const uint64_t q[2], int width, void *stream) {
    MQ_TRACE("mod_vsub");
    return blas(OP_VSUB, c, a, b, n, q, width, nullptr, stream);
}
extern "C" int mod_vmul(void *c, const void *a, const void *b, size_t n, const uint64_t q[2], int width, void *stream) {
    MQ_TRACE("mod_vmul");
    return blas(OP_VMUL, c, a, b, n, q, width, nullptr, stream);
}
extern "C" int mod_axpy(void *y, const uint64_t a[2], const void *x, size_t n, const uint64_t q[2], int width,
                        void *stream) {
    MQ_TRACE("mod_axpy");
    // y = a*x + y: the kernel's first operand is x, the second (and the output) is y
    return blas(OP_AXPY, y, x, y, n, q, width, a, stream);
}

// common.cuh -- types shared by the library's translation units (not part of the public ABI).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "residue.cuh"

namespace mq {

// A twiddle factor and its Shoup companion.
struct Tw64 {
    uint64_t w, wp;
};
struct __align__(16) Tw128 {
    uint4 w, wp;
};

// Where a tile's residues live in global memory (see ntt.cu).
enum Layout : int {
    LAYOUT_COL = 0,  // tile = column c of the N1 x N2 view: element l at l * N2 + c
    LAYOUT_ROW = 1,  // tile = row h: element l at h * N2 + l
    LAYOUT_NAT = 2,  // tile = row h of the bit-reversed view, addressed in natural order:
                     // element l at brv_L2(l) * N1 + brv_L1(h)
};

// Arguments of one pass of the transform over a batch of polynomials.
struct PassArgs {
    const void *in;      // source residues
    void *out;           // destination residues (may equal in)
    const void *tw;      // twiddle table (N entries, forward or inverse)
    uint64_t q[4];       // modulus, low word first (words beyond the residue width are zero)
    uint64_t sc[4], scp[4];  // N^-1 and its Shoup companion (inverse, global stage 0)
    uint64_t ws[4], wsp[4];  // twiddle[1] * N^-1 and its Shoup companion
    size_t in_stride;    // residues between consecutive polynomials in `in`
    size_t out_stride;   // ... in `out`
    unsigned long long batch;  // polynomials
    int logN;            // log2 of the transform size
    int L1;              // log2 N1 (rows of the N1 x N2 view)
    int col;             // 1: this pass works on columns (tiles of N1 residues), 0: rows (N2)
    int perm;            // rows only: tiles are picked so that brv_L1(h) is contiguous (natural order)
    int in_layout, out_layout;
    int scale;           // inverse only: fold N^-1 into global stage 0
    int final;           // last pass of the transform: store canonical residues
};

// The TMA form of a pass (tma.cuh): 128-bit residues, tiles of 2^TMA_L, each CTA group of 8 tiles
// moved by one tensor copy each way.
constexpr int TMA_L = 8;

// Whether a pass of tiles of 2^TMA_L over 128-bit residues can take the TMA form: both sides in the
// column view or both in the unpermuted row view, at least one group of 8 tiles per polynomial
// (groups never straddle polynomials), and coordinates that fit 32 bits.
inline bool tma_eligible(const PassArgs &a) {
    if (a.batch == 0 || a.batch >= (1ull << 31)) return false;
    if (a.col) return a.in_layout == LAYOUT_COL && a.out_layout == LAYOUT_COL && a.L1 == TMA_L && a.logN - a.L1 >= 3;
    return a.in_layout == LAYOUT_ROW && a.out_layout == LAYOUT_ROW && !a.perm && a.logN - a.L1 == TMA_L && a.L1 >= 3;
}

// Tensor map of one side of a TMA pass (host; ntt.cu).  col: the column view, else the row view.
// Returns 0, or nonzero when the driver refuses the map (the pass then takes the cp.async form).
int tile_map(CUtensorMap *m, bool col, const void *base, int logN, int L1, unsigned long long batch, size_t stride);

// Launch one pass; returns a cudaError_t.  L = log2 of the tile size, inv = direction.
cudaError_t launch_ntt_pass(int width, int L, bool inv, const PassArgs &a, cudaStream_t s);

// The Barrett constants of a plan's modulus, for the pointwise product of the fused polynomial
// product (see polymul.cuh).
struct MulArgs {
    uint64_t q[2], mu[2];
    int L;  // bit length of q
};

// Launch the fused pass of the polynomial product on tiles of 2^L residues: forward rounds of fa
// (a's tiles) and fb (b's tiles), pointwise product, inverse rounds and store of ia.
cudaError_t launch_polymul(int width, int L, const PassArgs &fa, const PassArgs &fb, const PassArgs &ia,
                           const MulArgs &m, cudaStream_t s);

// Build twiddle tables on the device (see ntt.cu).
cudaError_t launch_twiddle_build(int width, int logN, int cyclic, const uint64_t q[2], const uint64_t root[2],
                                 const uint64_t root_inv[2], const uint64_t mu[2], int L, void *tw_fwd,
                                 void *tw_inv, cudaStream_t s);

// Element-wise BLAS (see blas.cu).
enum BlasOp : int { OP_VADD = 0, OP_VSUB = 1, OP_VMUL = 2, OP_AXPY = 3 };
struct BlasArgs {
    void *c;
    const void *a, *b;
    size_t n;
    uint64_t q[2], mu[2];
    int L;
    uint64_t s[2], sp[2];  // axpy scalar and its Shoup companion
};
cudaError_t launch_blas(int width, int op, const BlasArgs &a, cudaStream_t s);

// The same operations on residues of three and four 64-bit words (see blas_wide.cu).
struct BlasWideArgs {
    void *c;
    const void *a, *b;
    size_t n;
    uint64_t q[4], mu[4];
    int L;
    uint64_t s[4], sp[4];  // axpy scalar and its Shoup companion
};
cudaError_t launch_blas_wide(int width, int op, const BlasWideArgs &a, cudaStream_t s);

}  // namespace mq

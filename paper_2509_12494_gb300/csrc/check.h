// check.h -- the input range check of MQ_CHECK_INPUTS (check.cu), internal to the library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mqntt.h"

namespace mq {

// One operand to check: `polys` runs of `n` residues, `stride` residues apart, of `width` words each,
// against the modulus q (width words, low first).
struct CheckRec {
    const void *p;
    unsigned long long polys, n, stride;
    int width;
    uint64_t q[4];
    const char *name;  // for the error message (host side only)
};

CheckRec check_rec(const void *p, unsigned long long polys, unsigned long long n, unsigned long long stride, int width,
                   const uint64_t *q, const char *name);

// Check operands on `s`, then synchronise `s`: MQ_OK, or MQ_ERR_RANGE naming the first operand that
// holds a residue >= q (message set).  Takes one word of stream-ordered scratch from the pool.
int range_check(const CheckRec *recs, int nrec, cudaStream_t s);

// The batched form's check (asynchronous, in the batch's graph after the counter reset): on a
// residue >= q it sets the status word ctrs[1] to MQ_ERR_RANGE and the item counter ctrs[0] to
// n_items.  d_recs is a device array of nrec records; max_residues sizes the grid.
cudaError_t launch_batch_check(const CheckRec *d_recs, unsigned nrec, unsigned long long max_residues, unsigned *dctrs,
                               unsigned n_items, cudaStream_t s);

}  // namespace mq

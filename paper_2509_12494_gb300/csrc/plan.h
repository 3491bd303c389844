// plan.h -- the layout of an ntt_plan (internal to the library).
#pragma once
#include <stdint.h>

struct ntt_plan {
    int device;
    unsigned log2n;
    int width;
    unsigned flags;
    uint64_t q[2], mu[2];
    int L;  // bit length of q
    uint64_t root[2], root_inv[2];
    void *tw_fwd, *tw_inv;  // N entries of (w, w') each
    uint64_t sc[2], scp[2], ws[2], wsp[2];
    int L1;  // rows of the N1 x N2 split (0: single pass)
};

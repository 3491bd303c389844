// plan.h -- the layout of an ntt_plan (internal to the library).
#pragma once
#include <stdint.h>

struct ntt_plan {
    int device;
    unsigned log2n;
    int width;
    unsigned flags;
    uint64_t q[4], mu[4];  // low word first; residues of up to four 64-bit words
    int L;  // bit length of q
    uint64_t root[4], root_inv[4];
    void *tw_fwd, *tw_inv;  // N entries of (w, w') each
    uint64_t sc[4], scp[4], ws[4], wsp[4];
    int L1;  // rows of the N1 x N2 split (0: single pass)
};

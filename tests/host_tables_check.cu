// Host-side rules of the batched form and the TMA form, checked without a GPU (built and run by
// tests/test_host_tables.py): which passes take the TMA form, the work items' meta bits, the
// layout constraints of the job descriptors the kernels read tensor maps from, and the shared
// memory each persistent instantiation asks for.  Prints one line per failed check and exits
// with their count.
#include <stddef.h>
#include <stdio.h>
#include <string.h>

#include "batch_kernel.cuh"

using namespace mq;
using namespace mq::batch_detail;

static int failures = 0;
#define CHECK(...)                                                 \
    do {                                                           \
        if (!(__VA_ARGS__)) {                                      \
            printf("FAILED line %d: %s\n", __LINE__, #__VA_ARGS__); \
            ++failures;                                            \
        }                                                          \
    } while (0)

static PassArgs pass(int col, int in_layout, int out_layout, int perm, int logN, int L1, unsigned long long batch) {
    PassArgs a;
    memset(&a, 0, sizeof a);
    a.col = col;
    a.in_layout = in_layout;
    a.out_layout = out_layout;
    a.perm = perm;
    a.logN = logN;
    a.L1 = L1;
    a.batch = batch;
    return a;
}

int main() {
    // the TMA form: tiles of 2^8 (the column pass of an 8 + * split, the row pass of a * + 8 split),
    // both sides in the same unpermuted view, at least 8 tiles per polynomial, 32-bit coordinates
    CHECK(tma_eligible(pass(1, LAYOUT_COL, LAYOUT_COL, 0, 16, 8, 256)));
    CHECK(tma_eligible(pass(0, LAYOUT_ROW, LAYOUT_ROW, 0, 16, 8, 256)));
    CHECK(tma_eligible(pass(0, LAYOUT_ROW, LAYOUT_ROW, 0, 15, 7, 6)));   // 2^15 = 2^7 x 2^8: the row pass
    CHECK(!tma_eligible(pass(1, LAYOUT_COL, LAYOUT_COL, 0, 15, 7, 6)));  // ... not its column pass (2^7)
    CHECK(tma_eligible(pass(1, LAYOUT_COL, LAYOUT_COL, 0, 17, 8, 3)));   // 2^17 = 2^8 x 2^9: the column pass
    CHECK(!tma_eligible(pass(0, LAYOUT_ROW, LAYOUT_ROW, 0, 17, 8, 3)));  // ... not its row pass (2^9)
    CHECK(!tma_eligible(pass(0, LAYOUT_ROW, LAYOUT_ROW, 1, 16, 8, 1)));  // natural order: permuted rows
    CHECK(!tma_eligible(pass(0, LAYOUT_ROW, LAYOUT_NAT, 0, 16, 8, 1)));  // natural-order output
    CHECK(!tma_eligible(pass(0, LAYOUT_NAT, LAYOUT_ROW, 0, 16, 8, 1)));  // natural-order input
    CHECK(!tma_eligible(pass(1, LAYOUT_COL, LAYOUT_ROW, 0, 16, 8, 1)));  // mixed views
    CHECK(!tma_eligible(pass(0, LAYOUT_ROW, LAYOUT_ROW, 0, 10, 2, 1)));  // 4 rows per polynomial < 8
    CHECK(!tma_eligible(pass(1, LAYOUT_COL, LAYOUT_COL, 0, 10, 8, 1)));  // 4 columns per polynomial < 8
    CHECK(!tma_eligible(pass(0, LAYOUT_ROW, LAYOUT_ROW, 0, 8, 0, 16)));  // one pass (no split)
    CHECK(!tma_eligible(pass(1, LAYOUT_COL, LAYOUT_COL, 0, 16, 8, 0)));  // empty batch
    CHECK(!tma_eligible(pass(1, LAYOUT_COL, LAYOUT_COL, 0, 16, 8, 1ull << 31)));  // poly coordinate > 2^31 - 1
    CHECK(tma_eligible(pass(1, LAYOUT_COL, LAYOUT_COL, 0, 16, 8, (1ull << 31) - 1)));

    // work-item meta bits: kind, width, direction, copy form, tile log size, all distinct
    CHECK(item_meta(false, 2, true, 8, true) == (ITEM_W128 | ITEM_INV | ITEM_TMA | (8u << 4)));
    CHECK(item_meta(true, 1, false, 0) == ITEM_BLAS);
    CHECK((ITEM_BLAS | ITEM_W128 | ITEM_INV | ITEM_TMA) == 15u);
    CHECK((item_meta(false, 2, false, LMAX, true) >> 4) == (unsigned)LMAX);
    CHECK(item_meta(false, 2, false, LMAX, true) <= 0xFFFFu);  // fits the 16-bit field
    CHECK(sizeof(ItemDev) == 32);
    CHECK(VARIANT_TMA_ONLY == (2 | 8));

    // tensor maps inside the job descriptors: aligned (the copy engine wants 64 bytes; the type
    // carries 128) in every element of a device array
    CHECK(sizeof(CUtensorMap) == 128 && alignof(CUtensorMap) == 128);
    CHECK(offsetof(JobDev, tm) % 128 == 0);
    CHECK(sizeof(JobDev) % 128 == 0);
    CHECK(alignof(JobDev) >= 128);

    // a TMA group: 8 tiles of 2^8 128-bit residues = 32 KiB, one warp per tile
    CHECK((ntt_detail::Shape<2, TMA_L>::G == 8 && ntt_detail::Shape<2, TMA_L>::T == 256));
    CHECK(ntt_detail::TMA_GROUP_BYTES == 32768u);

    // shared memory of the persistent instantiations: the prefetching form with 128-bit transforms
    // gets 1024-byte multiples covering both a cp.async group and a TMA group, plus 1024 bytes to
    // align the first buffer; everything else is unchanged
    const size_t k2 = kernel_smem<2>(), k1 = kernel_smem<1>();
    const size_t b2 = buffer_bytes<1, 2>(k2);
    CHECK(b2 % 1024 == 0);
    CHECK(b2 >= k2 && b2 >= ntt_detail::TMA_GROUP_BYTES && b2 < k2 + 1024);
    CHECK(dynamic_bytes<1, 2>(b2) == 2 * b2 + 1024);
    CHECK(buffer_bytes<0, 2>(k2) == k2 && dynamic_bytes<0, 2>(k2) == 2 * k2);
    CHECK(buffer_bytes<1, 1>(k1) == k1 && dynamic_bytes<1, 1>(k1) == 2 * k1);
    CHECK(3 * (dynamic_bytes<1, 2>(b2) + 1024) <= 228 * 1024);  // three CTAs per SM still fit

    if (failures) printf("%d failed\n", failures);
    else printf("ok\n");
    return failures;
}

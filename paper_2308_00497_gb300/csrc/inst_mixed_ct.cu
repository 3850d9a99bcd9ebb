// Per-length mixed-radix kernels (fftc_mixed_ct.cuh), FP32, for the lengths of the
// mixed-radix workload: (kind, L, lines per tile, threads, pitch, radices) exactly as the
// planner chooses them for these n, so the host can swap the runtime-radix kernel out.
//   single pass  n = 12, 96, 360, 1000, 3072, 6000
//   two passes   n = 10^4 (100 x 100), 3^10 (243 x 243), 10^5 (250 x 400), 10^6 (1000 x 1000)
#include "fftc_mixed_ct.cuh"

namespace fftc {

#define CT_ROWS(NT, L, C, ...)                                                               \
    mixed_ct_entry<KIND_ROWS, LAYOUT_IL, LAYOUT_IL, NT, L, C, L, __VA_ARGS__>(),             \
        mixed_ct_entry<KIND_ROWS, LAYOUT_SPLIT, LAYOUT_SPLIT, NT, L, C, L, __VA_ARGS__>()
#define CT_COLS(NT, L, C, P, ...)                                                            \
    mixed_ct_entry<KIND_COLS, LAYOUT_IL, LAYOUT_IL, NT, L, C, P, __VA_ARGS__>(),             \
        mixed_ct_entry<KIND_COLS, LAYOUT_SPLIT, LAYOUT_IL, NT, L, C, P, __VA_ARGS__>()
#define CT_ROWST(NT, L, C, P, ...)                                                           \
    mixed_ct_entry<KIND_ROWST, LAYOUT_IL, LAYOUT_IL, NT, L, C, P, __VA_ARGS__>(),            \
        mixed_ct_entry<KIND_ROWST, LAYOUT_IL, LAYOUT_SPLIT, NT, L, C, P, __VA_ARGS__>()

static const MixedCtEntry kMixedCtTable[] = {
    CT_ROWS(256, 12, 340, 12),
    CT_ROWS(256, 96, 40, 6, 16),
    CT_ROWS(256, 360, 8, 15, 3, 8),
    CT_ROWS(256, 1000, 4, 5, 5, 5, 8),
    CT_ROWS(256, 3072, 1, 12, 16, 16),
    CT_ROWS(512, 6000, 1, 15, 5, 5, 16),
    CT_COLS(256, 100, 40, 101, 5, 5, 4),
    CT_COLS(256, 243, 16, 243, 9, 9, 3),
    CT_COLS(256, 250, 16, 251, 10, 5, 5),
    CT_COLS(256, 1000, 4, 1001, 5, 5, 5, 8),
    CT_ROWST(256, 100, 40, 101, 5, 5, 4),
    CT_ROWST(256, 243, 16, 243, 9, 9, 3),
    CT_ROWST(256, 400, 10, 401, 5, 5, 16),
    CT_ROWST(256, 1000, 4, 1001, 5, 5, 5, 8),
};

const MixedCtEntry *find_mixed_ct(int kind, int lin, int lout, int nt, int L, int C, int pitch, int nst,
                                  const int8_t *radix) {
    for (const MixedCtEntry &e : kMixedCtTable) {
        if (e.kind != kind || e.lin != lin || e.lout != lout || e.nt != nt || e.L != L || e.C != C ||
            e.pitch != pitch || e.nst != nst)
            continue;
        bool same = true;
        for (int s = 0; s < nst; ++s) same = same && e.radix[s] == radix[s];
        if (same) return &e;
    }
    return nullptr;
}

}  // namespace fftc

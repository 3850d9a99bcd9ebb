// Instantiations of pipelined passes whose refill is issued after the tile's last
// shared read (fftc_pipe.cuh, EARLY), split layout: single pass n = 2^11 .. 2^14 (at 2^14
// one 135 KB tile per SM, at 2^13 two 68 KB tiles), four-step pass 2 (one bulk copy per
// tile) and four-step pass 1 (tensor-map boxes of 8, 16 or 32 columns, one landing buffer).
#include "fftc_pipe.cuh"

namespace fftc {

#define PRE(LOGL, LOGE, C, NBUF) pipe_entry<LOGL, LOGE, C, KIND_ROWS, LAYOUT_SPLIT, LAYOUT_SPLIT, 0, NBUF, true>()
#define PCE(LOGL, LOGE, C, LOGX, NBUF) pipe_entry<LOGL, LOGE, C, KIND_COLS, LAYOUT_SPLIT, LAYOUT_IL, LOGX, NBUF, true>()
#define PTE(LOGL, LOGE, C, LOGX, NBUF) pipe_entry<LOGL, LOGE, C, KIND_ROWST, LAYOUT_IL, LAYOUT_SPLIT, LOGX, NBUF, true>()

extern const KernelEntry kPipeEarlySplitTable[] = {
    PRE(11, 5, 2, 2),     PRE(12, 4, 1, 1),     PRE(12, 4, 1, 2),     PRE(13, 5, 1, 1),     PRE(13, 5, 1, 2),
    PRE(14, 5, 1, 1),     PRE(12, 5, 1, 1),
    PTE(8, 4, 16, 7, 2),  PTE(8, 4, 16, 8, 2),  PTE(9, 5, 8, 8, 2),   PTE(10, 5, 8, 8, 2),  PTE(10, 5, 8, 9, 2),
    PTE(10, 5, 8, 10, 2),
    // 16-row tiles (16 consecutive outputs per plane and store) for n = 2^17 .. 2^19
    PTE(9, 5, 16, 8, 1),  PTE(10, 5, 16, 8, 1), PTE(10, 5, 16, 9, 1),
    PCE(7, 4, 16, 8, 1),  PCE(8, 4, 16, 8, 1),  PCE(8, 4, 16, 9, 1),  PCE(8, 4, 32, 10, 1), PCE(9, 4, 16, 10, 1),
    // n = 2^20 as 2^9 x 2^11 and 2^10 x 2^10: 16 or 32 columns, 8 to 16 elements per thread
    PCE(9, 4, 16, 11, 1), PCE(9, 4, 32, 11, 1), PCE(10, 4, 16, 10, 1), PCE(10, 5, 8, 10, 1),
    // 32-column boxes for n = 2^15 .. 2^17
    PCE(7, 4, 32, 8, 1), PCE(8, 4, 32, 8, 1), PCE(8, 4, 32, 9, 1), PCE(9, 4, 32, 10, 1),
};
extern const int kPipeEarlySplitCount = sizeof(kPipeEarlySplitTable) / sizeof(kPipeEarlySplitTable[0]);

}  // namespace fftc

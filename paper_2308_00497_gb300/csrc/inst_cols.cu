// Instantiations of four-step pass 1 (KIND_COLS): column FFTs of length M = 2^LOGL at
// stride K = 2^LOGX, C adjacent columns per CTA, output interleaved into the workspace.
// One instance per n = 2^14 .. 2^20 with the stride compile-time, plus runtime-stride ones.
#include "fftc_pass.cuh"

namespace fftc {

#define C2(LOGL, LOGE, C, LOGX) entry<LOGL, LOGE, C, KIND_COLS, LAYOUT_IL, LAYOUT_IL, LOGX>(), \
                                entry<LOGL, LOGE, C, KIND_COLS, LAYOUT_SPLIT, LAYOUT_IL, LOGX>()

extern const KernelEntry kColsTable[] = {
    // n = 2^14 .. 2^20 (M x K = 7x7, 7x8, 8x8, 8x9, 8x10, 9x10, 10x10), and 9x9
    C2(7, 4, 16, 7), C2(7, 4, 16, 8), C2(8, 4, 16, 8), C2(8, 4, 16, 9), C2(8, 4, 32, 10), C2(9, 4, 16, 10),
    C2(10, 5, 8, 10), C2(9, 4, 16, 9),
    // 2^20 split as 2^9 x 2^11 with the stride at compile time
    C2(9, 4, 16, 11), C2(9, 5, 16, 11),
    // 32-column bands (128-byte rows in each plane of the split layout) for n = 2^15 .. 2^17
    C2(7, 4, 32, 8), C2(8, 4, 32, 8), C2(8, 4, 32, 9), C2(8, 5, 32, 8), C2(8, 5, 32, 9),
    C2(9, 5, 32, 10), C2(9, 5, 32, 11),
    // runtime strides (tuning alternatives)
    C2(6, 4, 16, 0), C2(7, 4, 16, 0), C2(8, 4, 16, 0), C2(9, 4, 16, 0), C2(9, 5, 16, 0), C2(10, 4, 16, 0),
    C2(10, 5, 16, 0), C2(9, 5, 8, 0), C2(10, 5, 8, 0), C2(10, 4, 8, 0),
};
extern const int kColsCount = sizeof(kColsTable) / sizeof(kColsTable[0]);

}  // namespace fftc

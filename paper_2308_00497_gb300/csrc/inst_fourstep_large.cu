// Instantiations of the four-step passes for n = 2^21 .. 2^24, where Eq. 1 applied once at
// the HBM level needs a factor above 2^10: column FFTs of length M = 2^11 or 2^12 (pass 1,
// KIND_COLS) and transposed-row FFTs of length K = 2^11 or 2^12 (pass 2, KIND_ROWST), the
// other factor a run-time stride. A tile holds 8 lines of 2^11 or 4 lines of 2^12 points
// (about 132 KB of shared memory, one CTA per SM of 512 threads with 32 elements each or 1024
// with 16), or 4 lines of 2^11 (66 KB, up to three CTAs per SM), so every column access still
// covers at least one whole 32-byte sector.
#include "fftc_pass.cuh"

namespace fftc {

#define LC(LOGL, LOGE, C) entry<LOGL, LOGE, C, KIND_COLS, LAYOUT_IL, LAYOUT_IL, 0>(), \
                          entry<LOGL, LOGE, C, KIND_COLS, LAYOUT_SPLIT, LAYOUT_IL, 0>()
#define LT(LOGL, LOGE, C) entry<LOGL, LOGE, C, KIND_ROWST, LAYOUT_IL, LAYOUT_IL, 0>(), \
                          entry<LOGL, LOGE, C, KIND_ROWST, LAYOUT_IL, LAYOUT_SPLIT, 0>()

// three-pass 2^24 (n = 2^8 x 2^8 x 2^8): pass 1 columns of 256 at the element stride 2^16
// (16 or 32 columns a tile) and pass 3 rows of 256 stored at the stride 2^16, at compile time
#define LCX(LOGL, LOGE, C, LOGX) entry<LOGL, LOGE, C, KIND_COLS, LAYOUT_IL, LAYOUT_IL, LOGX>(), \
                                 entry<LOGL, LOGE, C, KIND_COLS, LAYOUT_SPLIT, LAYOUT_IL, LOGX>()
#define LTX(LOGL, LOGE, C, LOGX) entry<LOGL, LOGE, C, KIND_ROWST, LAYOUT_IL, LAYOUT_IL, LOGX>(), \
                                 entry<LOGL, LOGE, C, KIND_ROWST, LAYOUT_IL, LAYOUT_SPLIT, LOGX>()

extern const KernelEntry kLargeTable[] = {
    LC(11, 5, 8), LC(12, 5, 4), LC(11, 4, 8), LC(11, 5, 4), LC(12, 4, 4),
    LT(11, 5, 8), LT(12, 5, 4), LT(11, 4, 8), LT(11, 5, 4), LT(12, 4, 4),
    LCX(8, 4, 16, 16), LCX(8, 4, 32, 16), LTX(8, 4, 16, 16),
};
extern const int kLargeCount = sizeof(kLargeTable) / sizeof(kLargeTable[0]);

}  // namespace fftc

// Instantiations of the single-pass kernel (KIND_ROWS, split layout): one HBM round
// trip per transform. Lines per CTA = max(1, 256 / (L / E)) so that a CTA has 256 threads.
#include "fftc_pass.cuh"

namespace fftc {

#define ROWS_C(LOGL, LOGE) ((1 << ((LOGL) - (LOGE))) >= 256 ? 1 : 256 / (1 << ((LOGL) - (LOGE))))
#define R1(LOGL, LOGE) entry<LOGL, LOGE, ROWS_C(LOGL, LOGE), KIND_ROWS, LAYOUT_SPLIT, LAYOUT_SPLIT>()
#define T1(LOGL) entry<LOGL, LOGL, 128, KIND_ROWS, LAYOUT_SPLIT, LAYOUT_SPLIT>()

extern const KernelEntry kRowsSplitTable[] = {
    T1(1), T1(2), T1(3), T1(4),
    R1(5, 4), R1(6, 4), R1(7, 4), R1(8, 4),
    R1(9, 4), R1(9, 5), R1(10, 4), R1(10, 5), R1(11, 4), R1(11, 5),
    R1(12, 4), R1(12, 5), R1(13, 4), R1(13, 5), R1(14, 4), R1(14, 5),
};
extern const int kRowsSplitCount = sizeof(kRowsSplitTable) / sizeof(kRowsSplitTable[0]);

}  // namespace fftc

// Instantiations of the column pass with split planes in and out (runtime element stride):
// the strided axes of split-layout multidimensional arrays with power-of-two lengths
// 64..1024 (the four-step pass 1 writes the interleaved workspace instead, inst_cols.cu).
#include "fftc_pass.cuh"

namespace fftc {

#define CS(LOGL, LOGE, C) entry<LOGL, LOGE, C, KIND_COLS, LAYOUT_SPLIT, LAYOUT_SPLIT, 0>()

extern const KernelEntry kColsSplitTable[] = {
    CS(6, 4, 16), CS(7, 4, 16), CS(8, 4, 16), CS(9, 4, 16), CS(10, 5, 8),
};
extern const int kColsSplitCount = sizeof(kColsSplitTable) / sizeof(kColsSplitTable[0]);

}  // namespace fftc

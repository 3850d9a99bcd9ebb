// Instantiations of four-step pass 1 (KIND_COLS): column FFTs of length M at stride K,
// 16 adjacent columns per CTA, output interleaved into the workspace.
#include "fftc_pass.cuh"

namespace fftc {

#define C2(LOGL, LOGE) entry<LOGL, LOGE, 16, KIND_COLS, LAYOUT_IL, LAYOUT_IL>(), \
                       entry<LOGL, LOGE, 16, KIND_COLS, LAYOUT_SPLIT, LAYOUT_IL>()
#define C8(LOGL, LOGE) entry<LOGL, LOGE, 8, KIND_COLS, LAYOUT_IL, LAYOUT_IL>(), \
                       entry<LOGL, LOGE, 8, KIND_COLS, LAYOUT_SPLIT, LAYOUT_IL>()

extern const KernelEntry kColsTable[] = {
    C2(6, 4), C2(7, 4), C2(8, 4), C2(9, 4), C2(9, 5), C2(10, 4), C2(10, 5),
    C8(9, 5), C8(10, 5), C8(10, 4),
};
extern const int kColsCount = sizeof(kColsTable) / sizeof(kColsTable[0]);

}  // namespace fftc

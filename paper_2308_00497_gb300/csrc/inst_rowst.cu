// Instantiations of four-step pass 2 (KIND_ROWST): row FFTs of length K = 2^LOGL from the
// workspace, C adjacent rows per CTA, written transposed (stride M = 2^LOGX) in the user
// layout. One instance per n = 2^14 .. 2^20 with the stride compile-time, plus
// runtime-stride ones.
#include "fftc_pass.cuh"

namespace fftc {

#define T2(LOGL, LOGE, C, LOGX) entry<LOGL, LOGE, C, KIND_ROWST, LAYOUT_IL, LAYOUT_IL, LOGX>(), \
                                entry<LOGL, LOGE, C, KIND_ROWST, LAYOUT_IL, LAYOUT_SPLIT, LOGX>()

extern const KernelEntry kRowsTTable[] = {
    // n = 2^14 .. 2^20 (K x M = 7x7, 8x7, 8x8, 9x8, 10x8, 10x9, 10x10), and 9x9
    T2(7, 4, 16, 7), T2(8, 4, 16, 7), T2(8, 4, 16, 8), T2(9, 5, 8, 8), T2(10, 5, 8, 8), T2(10, 5, 8, 9),
    T2(10, 5, 8, 10), T2(9, 5, 8, 9),
    // runtime strides (tuning alternatives)
    T2(7, 4, 16, 0), T2(8, 4, 16, 0), T2(9, 4, 16, 0), T2(9, 5, 16, 0), T2(10, 4, 16, 0), T2(10, 5, 16, 0),
    T2(9, 5, 8, 0), T2(10, 5, 8, 0), T2(10, 4, 8, 0),
};
extern const int kRowsTCount = sizeof(kRowsTTable) / sizeof(kRowsTTable[0]);

}  // namespace fftc

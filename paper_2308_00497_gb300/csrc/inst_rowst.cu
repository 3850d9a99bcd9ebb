// Instantiations of four-step pass 2 (KIND_ROWST): row FFTs of length K from the
// workspace, 16 adjacent rows per CTA, written transposed (stride M) in the user layout.
#include "fftc_pass.cuh"

namespace fftc {

#define T2(LOGL, LOGE) entry<LOGL, LOGE, 16, KIND_ROWST, LAYOUT_IL, LAYOUT_IL>(), \
                       entry<LOGL, LOGE, 16, KIND_ROWST, LAYOUT_IL, LAYOUT_SPLIT>()

#define T8(LOGL, LOGE) entry<LOGL, LOGE, 8, KIND_ROWST, LAYOUT_IL, LAYOUT_IL>(), \
                       entry<LOGL, LOGE, 8, KIND_ROWST, LAYOUT_IL, LAYOUT_SPLIT>()

extern const KernelEntry kRowsTTable[] = {
    T2(7, 4), T2(8, 4), T2(9, 4), T2(9, 5), T2(10, 4), T2(10, 5),
    T8(9, 5), T8(10, 5), T8(10, 4),
};
extern const int kRowsTCount = sizeof(kRowsTTable) / sizeof(kRowsTTable[0]);

}  // namespace fftc

// Instantiations of the runtime-radix kernel (four-step pass 2, FP64); the host picks them from
// these tables (fftc_mixed.cu). One unit per table keeps the compile parallel.
// FP64 tiles never exceed 4096 elements, so the 512-thread variants are not built.
#include "fftc_mixed.cuh"

namespace fftc {

// transposed rows (four-step pass 2): interleaved or split output
extern const MixedKernel kMixedRowsTF64[2][2] = {
    {&k_mixed<KIND_ROWST, LAYOUT_IL, LAYOUT_IL, 256, double2>, nullptr},
    {&k_mixed<KIND_ROWST, LAYOUT_IL, LAYOUT_SPLIT, 256, double2>, nullptr},
};

}  // namespace fftc

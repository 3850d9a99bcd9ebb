// Instantiations of the runtime-radix kernel (single pass, FP64); the host picks them from
// these tables (fftc_mixed.cu). One unit per table keeps the compile parallel.
// FP64 tiles never exceed 4096 elements, so the 512-thread variants are not built.
#include "fftc_mixed.cuh"

namespace fftc {

extern const MixedKernel kMixedRowsF64[2][2] = {
    {&k_mixed<KIND_ROWS, LAYOUT_IL, LAYOUT_IL, 256, double2>, nullptr},
    {&k_mixed<KIND_ROWS, LAYOUT_SPLIT, LAYOUT_SPLIT, 256, double2>, nullptr},
};

}  // namespace fftc

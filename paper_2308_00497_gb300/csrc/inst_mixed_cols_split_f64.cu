// Instantiations of the runtime-radix kernel (four-step pass 1 and strided axes, split input, FP64); the host picks them from
// these tables (fftc_mixed.cu). One unit per table keeps the compile parallel.
// FP64 tiles never exceed 4096 elements, so the 512-thread variants are not built.
#include "fftc_mixed.cuh"

namespace fftc {

// columns from split planes: into the interleaved workspace (four-step pass 1) or back into
// split planes (strided axes)
extern const MixedKernel kMixedColsSplitF64[2][2] = {
    {&k_mixed<KIND_COLS, LAYOUT_SPLIT, LAYOUT_IL, 256, double2>, nullptr},
    {&k_mixed<KIND_COLS, LAYOUT_SPLIT, LAYOUT_SPLIT, 256, double2>, nullptr},
};

}  // namespace fftc

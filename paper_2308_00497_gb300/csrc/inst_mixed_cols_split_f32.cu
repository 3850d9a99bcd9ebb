// Instantiations of the runtime-radix kernel (four-step pass 1 and strided axes, split input, FP32); the host picks them from
// these tables (fftc_mixed.cu). One unit per table keeps the compile parallel.
#include "fftc_mixed.cuh"

namespace fftc {

// columns from split planes: into the interleaved workspace (four-step pass 1) or back into
// split planes (strided axes)
extern const MixedKernel kMixedColsSplitF32[2][2] = {
    {&k_mixed<KIND_COLS, LAYOUT_SPLIT, LAYOUT_IL, 256, float2>, &k_mixed<KIND_COLS, LAYOUT_SPLIT, LAYOUT_IL, 512, float2>},
    {&k_mixed<KIND_COLS, LAYOUT_SPLIT, LAYOUT_SPLIT, 256, float2>, &k_mixed<KIND_COLS, LAYOUT_SPLIT, LAYOUT_SPLIT, 512, float2>},
};

}  // namespace fftc

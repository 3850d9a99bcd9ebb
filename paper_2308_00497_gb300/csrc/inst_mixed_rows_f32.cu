// Instantiations of the runtime-radix kernel (single pass, FP32); the host picks them from
// these tables (fftc_mixed.cu). One unit per table keeps the compile parallel.
#include "fftc_mixed.cuh"

namespace fftc {

extern const MixedKernel kMixedRowsF32[2][2] = {
    {&k_mixed<KIND_ROWS, LAYOUT_IL, LAYOUT_IL, 256, float2>, &k_mixed<KIND_ROWS, LAYOUT_IL, LAYOUT_IL, 512, float2>},
    {&k_mixed<KIND_ROWS, LAYOUT_SPLIT, LAYOUT_SPLIT, 256, float2>, &k_mixed<KIND_ROWS, LAYOUT_SPLIT, LAYOUT_SPLIT, 512, float2>},
};

}  // namespace fftc

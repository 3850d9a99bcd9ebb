// Instantiations of the runtime-radix kernel (four-step pass 2, FP32); the host picks them from
// these tables (fftc_mixed.cu). One unit per table keeps the compile parallel.
#include "fftc_mixed.cuh"

namespace fftc {

// transposed rows (four-step pass 2): interleaved or split output
extern const MixedKernel kMixedRowsTF32[2][2] = {
    {&k_mixed<KIND_ROWST, LAYOUT_IL, LAYOUT_IL, 256, float2>, &k_mixed<KIND_ROWST, LAYOUT_IL, LAYOUT_IL, 512, float2>},
    {&k_mixed<KIND_ROWST, LAYOUT_IL, LAYOUT_SPLIT, 256, float2>, &k_mixed<KIND_ROWST, LAYOUT_IL, LAYOUT_SPLIT, 512, float2>},
};

}  // namespace fftc

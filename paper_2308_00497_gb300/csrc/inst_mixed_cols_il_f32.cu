// Instantiations of the runtime-radix kernel (four-step pass 1 and strided axes, interleaved, FP32); the host picks them from
// these tables (fftc_mixed.cu). One unit per table keeps the compile parallel.
#include "fftc_mixed.cuh"

namespace fftc {

// columns, interleaved in and out (four-step pass 1, strided axes)
extern const MixedKernel kMixedColsIlF32[2] = {&k_mixed<KIND_COLS, LAYOUT_IL, LAYOUT_IL, 256, float2>,
                                              &k_mixed<KIND_COLS, LAYOUT_IL, LAYOUT_IL, 512, float2>};

}  // namespace fftc

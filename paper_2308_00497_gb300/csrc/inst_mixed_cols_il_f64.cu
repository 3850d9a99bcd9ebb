// Instantiations of the runtime-radix kernel (four-step pass 1 and strided axes, interleaved, FP64); the host picks them from
// these tables (fftc_mixed.cu). One unit per table keeps the compile parallel.
// FP64 tiles never exceed 4096 elements, so the 512-thread variants are not built.
#include "fftc_mixed.cuh"

namespace fftc {

// columns, interleaved in and out (four-step pass 1, strided axes)
extern const MixedKernel kMixedColsIlF64[2] = {&k_mixed<KIND_COLS, LAYOUT_IL, LAYOUT_IL, 256, double2>,
                                              nullptr};

}  // namespace fftc

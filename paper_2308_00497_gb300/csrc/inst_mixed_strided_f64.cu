// Instantiations of the runtime-radix kernel (four-step passes and strided axes, FP64); the host picks them from
// these tables (fftc_mixed.cu). One unit per table keeps the compile parallel.
#include "fftc_mixed.cuh"

namespace fftc {

// columns: il -> il, split -> il (four-step workspace), split -> split (strided axes);
// transposed rows: il -> il, il -> split
extern const MixedKernel kMixedStridedF64[5][2] = {
    {&k_mixed<KIND_COLS, LAYOUT_IL, LAYOUT_IL, 256, double2>, &k_mixed<KIND_COLS, LAYOUT_IL, LAYOUT_IL, 512, double2>},
    {&k_mixed<KIND_COLS, LAYOUT_SPLIT, LAYOUT_IL, 256, double2>, &k_mixed<KIND_COLS, LAYOUT_SPLIT, LAYOUT_IL, 512, double2>},
    {&k_mixed<KIND_COLS, LAYOUT_SPLIT, LAYOUT_SPLIT, 256, double2>,
     &k_mixed<KIND_COLS, LAYOUT_SPLIT, LAYOUT_SPLIT, 512, double2>},
    {&k_mixed<KIND_ROWST, LAYOUT_IL, LAYOUT_IL, 256, double2>, &k_mixed<KIND_ROWST, LAYOUT_IL, LAYOUT_IL, 512, double2>},
    {&k_mixed<KIND_ROWST, LAYOUT_IL, LAYOUT_SPLIT, 256, double2>, &k_mixed<KIND_ROWST, LAYOUT_IL, LAYOUT_SPLIT, 512, double2>},
};

}  // namespace fftc

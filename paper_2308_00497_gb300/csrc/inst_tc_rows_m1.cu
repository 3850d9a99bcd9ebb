// Single-pass tensor-core kernels, precision mode 1 (FP16); lists in fftc_tc_inst.cuh.
#include "fftc_tc_inst.cuh"

namespace fftc {

extern const KernelEntry kTcRowsM1Table[] = {FFTC_TC_ROWS(1, LAYOUT_IL), FFTC_TC_ROWS(1, LAYOUT_SPLIT)};
extern const int kTcRowsM1Count = sizeof(kTcRowsM1Table) / sizeof(kTcRowsM1Table[0]);

}  // namespace fftc

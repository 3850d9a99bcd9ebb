// Single-pass tensor-core kernels, precision mode 2 (BF16); lists in fftc_tc_inst.cuh.
#include "fftc_tc_inst.cuh"

namespace fftc {

extern const KernelEntry kTcRowsM2Table[] = {FFTC_TC_ROWS(2, LAYOUT_IL), FFTC_TC_ROWS(2, LAYOUT_SPLIT)};
extern const int kTcRowsM2Count = sizeof(kTcRowsM2Table) / sizeof(kTcRowsM2Table[0]);

}  // namespace fftc

// Single-pass tensor-core kernels, precision mode 3 (FP16 hi+lo split); lists in fftc_tc_inst.cuh.
#include "fftc_tc_inst.cuh"

namespace fftc {

extern const KernelEntry kTcRowsM3Table[] = {FFTC_TC_ROWS(3, LAYOUT_IL), FFTC_TC_ROWS(3, LAYOUT_SPLIT)};
extern const int kTcRowsM3Count = sizeof(kTcRowsM3Table) / sizeof(kTcRowsM3Table[0]);

}  // namespace fftc

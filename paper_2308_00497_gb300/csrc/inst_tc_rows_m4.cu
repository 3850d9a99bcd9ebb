// Single-pass tensor-core kernels, precision mode 4 (BF16 hi+lo split); lists in fftc_tc_inst.cuh.
#include "fftc_tc_inst.cuh"

namespace fftc {

extern const KernelEntry kTcRowsM4Table[] = {FFTC_TC_ROWS(4, LAYOUT_IL), FFTC_TC_ROWS(4, LAYOUT_SPLIT)};
extern const int kTcRowsM4Count = sizeof(kTcRowsM4Table) / sizeof(kTcRowsM4Table[0]);

}  // namespace fftc

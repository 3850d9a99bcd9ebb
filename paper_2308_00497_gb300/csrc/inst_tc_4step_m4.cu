// Four-step tensor-core passes, precision mode 4 (BF16 hi+lo split); lists in fftc_tc_inst.cuh.
#include "fftc_tc_inst.cuh"

namespace fftc {

extern const KernelEntry kTc4M4Table[] = {FFTC_TC_4STEP(4)};
extern const int kTc4M4Count = sizeof(kTc4M4Table) / sizeof(kTc4M4Table[0]);

}  // namespace fftc

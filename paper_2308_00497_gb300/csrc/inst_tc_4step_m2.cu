// Four-step tensor-core passes, precision mode 2 (BF16); lists in fftc_tc_inst.cuh.
#include "fftc_tc_inst.cuh"

namespace fftc {

extern const KernelEntry kTc4M2Table[] = {FFTC_TC_4STEP(2)};
extern const int kTc4M2Count = sizeof(kTc4M2Table) / sizeof(kTc4M2Table[0]);

}  // namespace fftc

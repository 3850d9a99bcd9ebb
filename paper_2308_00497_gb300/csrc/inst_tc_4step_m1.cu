// Four-step tensor-core passes, precision mode 1 (FP16); lists in fftc_tc_inst.cuh.
#include "fftc_tc_inst.cuh"

namespace fftc {

extern const KernelEntry kTc4M1Table[] = {FFTC_TC_4STEP(1)};
extern const int kTc4M1Count = sizeof(kTc4M1Table) / sizeof(kTc4M1Table[0]);

}  // namespace fftc

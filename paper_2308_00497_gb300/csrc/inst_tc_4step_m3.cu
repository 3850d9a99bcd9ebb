// Four-step tensor-core passes, precision mode 3 (FP16 hi+lo split); lists in fftc_tc_inst.cuh.
#include "fftc_tc_inst.cuh"

namespace fftc {

extern const KernelEntry kTc4M3Table[] = {FFTC_TC_4STEP(3)};
extern const int kTc4M3Count = sizeof(kTc4M3Table) / sizeof(kTc4M3Table[0]);

}  // namespace fftc

// Entry points of the extensions that are not part of this build yet.
#include "fftc_plan.h"

namespace fftc {
fftc_status plan_build_tc(fftc_plan_s *) { return FFTC_ERR_UNSUPPORTED_SIZE; }
fftc_status plan_run_tc(fftc_plan_s *, const void *, void *, cudaStream_t) { return FFTC_ERR_INVALID_PLAN; }
}  // namespace fftc

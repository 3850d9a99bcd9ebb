// Entry points of the extensions that are not part of this build yet.
#include "fftc_plan.h"

namespace fftc {
fftc_status plan_build_tc(fftc_plan_s *) { return FFTC_ERR_UNSUPPORTED_SIZE; }
fftc_status plan_run_tc(fftc_plan_s *, const void *, void *, cudaStream_t) { return FFTC_ERR_INVALID_PLAN; }
void plan_destroy_extra(fftc_plan_s *) {}
}  // namespace fftc

extern "C" fftc_plan fftc_plan_create_uneven(int64_t, const int64_t *, const int8_t *, const int64_t *, fftc_layout,
                                             fftc_precision) {
    return nullptr;
}

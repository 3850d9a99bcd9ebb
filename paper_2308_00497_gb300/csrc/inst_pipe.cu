// Instantiations of the pipelined persistent single-pass kernel (bulk-copy landing
// buffers, fftc_pipe.cuh) for n = 2^8 .. 2^13, both layouts. The first entry of each
// size is the default; the others are tuning alternatives.
#include "fftc_pipe.cuh"

namespace fftc {

#define PR2(LOGL, LOGE, C, NBUF) pipe_entry<LOGL, LOGE, C, LAYOUT_IL, NBUF>(), pipe_entry<LOGL, LOGE, C, LAYOUT_SPLIT, NBUF>()

extern const KernelEntry kPipeTable[] = {
    PR2(8, 4, 8, 3),  PR2(9, 5, 8, 2),  PR2(10, 5, 4, 2), PR2(11, 5, 2, 2), PR2(12, 4, 1, 2), PR2(13, 5, 1, 2),
    // alternatives
    PR2(9, 4, 4, 3),  PR2(10, 5, 8, 2), PR2(11, 4, 2, 2), PR2(12, 5, 1, 2), PR2(13, 4, 1, 2),
};
extern const int kPipeCount = sizeof(kPipeTable) / sizeof(kPipeTable[0]);

}  // namespace fftc

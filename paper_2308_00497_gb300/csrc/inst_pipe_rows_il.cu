// Instantiations of the pipelined persistent single-pass kernel (bulk-copy landing
// buffers, fftc_pipe.cuh) for n = 2^8 .. 2^13, one layout per unit. The first entry of
// each size is its default; the others are tuning alternatives.
#include "fftc_pipe.cuh"

namespace fftc {

#define PR1(LOGL, LOGE, C, NBUF) pipe_entry<LOGL, LOGE, C, KIND_ROWS, LAYOUT_IL, LAYOUT_IL, 0, NBUF>()

extern const KernelEntry kPipeRowsIlTable[] = {
    PR1(8, 4, 8, 3),  PR1(9, 5, 8, 2),  PR1(10, 5, 4, 2), PR1(11, 5, 2, 2), PR1(12, 4, 1, 2), PR1(13, 5, 1, 2),
    // alternatives
    PR1(9, 4, 4, 3),  PR1(10, 5, 8, 2), PR1(11, 4, 2, 2), PR1(12, 5, 1, 2), PR1(13, 4, 1, 2),
};
extern const int kPipeRowsIlCount = sizeof(kPipeRowsIlTable) / sizeof(kPipeRowsIlTable[0]);

}  // namespace fftc

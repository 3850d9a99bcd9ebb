// Instantiations of the single-pass kernels whose radix-16 stages run on the tensor
// cores (fftc_tc.cuh; the precision mode is a run-time argument): n = 2^7, 2^8 as plain
// CTAs of 256 threads, n = 2^9 .. 2^14 as persistent kernels fed by bulk copies (two
// landing buffers up to 2^12, one above), 16 elements per thread, both layouts.
#include "fftc_pipe.cuh"

namespace fftc {

#define TR(LOGL, C, LAY) entry<LOGL, 4, C, KIND_ROWS, LAY, LAY, 0, true>()
#define TP(LOGL, C, NBUF, LAY) pipe_entry<LOGL, 4, C, KIND_ROWS, LAY, LAY, 0, NBUF, true, true>()
#define TCROWS(LAY)                                                                                          \
    TR(7, 32, LAY), TR(8, 16, LAY), TP(9, 8, 2, LAY), TP(10, 4, 2, LAY), TP(11, 2, 2, LAY), TP(12, 1, 2, LAY), \
        TP(13, 1, 1, LAY), TP(14, 1, 1, LAY)

extern const KernelEntry kTcRowsTable[] = {TCROWS(LAYOUT_IL), TCROWS(LAYOUT_SPLIT)};
extern const int kTcRowsCount = sizeof(kTcRowsTable) / sizeof(kTcRowsTable[0]);

}  // namespace fftc

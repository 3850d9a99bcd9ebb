// Pipelined four-step pass 2 (KIND_ROWST) for n = 2^21 .. 2^24 (fftc_pipe.cuh): one bulk copy
// per tile of C consecutive workspace rows of length 2^11 or 2^12, the transposed store at a
// run-time stride; and for 2^20 split as 2^9 x 2^11, rows of 2^11 with the store stride 2^9 at
// compile time. The 132 KB tiles have one landing buffer with the refill issued after the
// last shared read; the 66 KB tiles (4 rows of 2^11) have two.
#include "fftc_pipe.cuh"

namespace fftc {

#define PTL(LOGL, LOGE, C, NBUF, EARLY)                                                    \
    pipe_entry<LOGL, LOGE, C, KIND_ROWST, LAYOUT_IL, LAYOUT_IL, 0, NBUF, EARLY>(),         \
        pipe_entry<LOGL, LOGE, C, KIND_ROWST, LAYOUT_IL, LAYOUT_SPLIT, 0, NBUF, EARLY>()

// the same with the transposed-store stride M = 2^LOGX at compile time
#define PTLX(LOGL, LOGE, C, LOGX, NBUF, EARLY)                                             \
    pipe_entry<LOGL, LOGE, C, KIND_ROWST, LAYOUT_IL, LAYOUT_IL, LOGX, NBUF, EARLY>(),      \
        pipe_entry<LOGL, LOGE, C, KIND_ROWST, LAYOUT_IL, LAYOUT_SPLIT, LOGX, NBUF, EARLY>()

extern const KernelEntry kPipeLargeTable[] = {
    PTL(11, 5, 8, 1, true),
    PTLX(11, 5, 8, 9, 1, true),   // 2^20 as 2^9 x 2^11
    PTL(12, 5, 4, 1, true),
    PTL(11, 5, 4, 2, true),
};
extern const int kPipeLargeCount = sizeof(kPipeLargeTable) / sizeof(kPipeLargeTable[0]);

}  // namespace fftc

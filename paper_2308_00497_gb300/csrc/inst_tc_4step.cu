// Instantiations of the four-step passes (n = M K, Eq. 1 at the memory level) whose
// radix-16 stages run on the tensor cores: n = 2^15 (M = 2^7, K = 2^8) and 2^16 (M = K =
// 2^8), 16 lines per tile, 16 elements per thread. Pass 1 reads columns with plain loads
// (with an L2 prefetch of the CTA's next tile) or tensor-map boxes into one landing buffer;
// pass 2 reads rows with plain loads or one bulk copy per tile into two landing buffers,
// and writes them transposed.
#include "fftc_pipe.cuh"

namespace fftc {

#define TCOL(LOGM, LOGK)                                                                   \
    entry<LOGM, 4, 16, KIND_COLS, LAYOUT_IL, LAYOUT_IL, LOGK, true>(),                   \
        pipe_entry<LOGM, 4, 16, KIND_COLS, LAYOUT_IL, LAYOUT_IL, LOGK, 1, true, true>(),  \
        pipe_entry<LOGM, 4, 16, KIND_COLS, LAYOUT_SPLIT, LAYOUT_IL, LOGK, 1, true, true>()
#define TROW(LOGK, LOGM)                                                                   \
    entry<LOGK, 4, 16, KIND_ROWST, LAYOUT_IL, LAYOUT_IL, LOGM, true>(),                  \
        entry<LOGK, 4, 16, KIND_ROWST, LAYOUT_IL, LAYOUT_SPLIT, LOGM, true>(),           \
        pipe_entry<LOGK, 4, 16, KIND_ROWST, LAYOUT_IL, LAYOUT_IL, LOGM, 2, true, true>(), \
        pipe_entry<LOGK, 4, 16, KIND_ROWST, LAYOUT_IL, LAYOUT_SPLIT, LOGM, 2, true, true>()

extern const KernelEntry kTc4Table[] = {TCOL(7, 8), TCOL(8, 8), TROW(8, 7), TROW(8, 8)};
extern const int kTc4Count = sizeof(kTc4Table) / sizeof(kTc4Table[0]);

}  // namespace fftc

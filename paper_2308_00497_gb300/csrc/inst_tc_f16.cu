// Instantiations of the tensor-core radix-16 passes with FP16 operands (plain and hi+lo
// split): single pass for 2^7 <= n <= 2^13 (lines per CTA = max(1, 4096 / n)), and the
// two four-step passes for n = 2^14 .. 2^16 (16 lines per CTA).
#include "fftc_tc.cuh"

namespace fftc {

#define TCR(LOGL, PREC)                                                                             \
    tc_entry<LOGL, ((1 << LOGL) >= 4096 ? 1 : 4096 >> LOGL), KIND_ROWS, LAYOUT_IL, LAYOUT_IL, PREC>(), \
        tc_entry<LOGL, ((1 << LOGL) >= 4096 ? 1 : 4096 >> LOGL), KIND_ROWS, LAYOUT_SPLIT, LAYOUT_SPLIT, PREC>()
#define TC4(LOGL, PREC)                                                  \
    tc_entry<LOGL, 16, KIND_COLS, LAYOUT_IL, LAYOUT_IL, PREC>(),         \
        tc_entry<LOGL, 16, KIND_COLS, LAYOUT_SPLIT, LAYOUT_IL, PREC>(),  \
        tc_entry<LOGL, 16, KIND_ROWST, LAYOUT_IL, LAYOUT_IL, PREC>(),    \
        tc_entry<LOGL, 16, KIND_ROWST, LAYOUT_IL, LAYOUT_SPLIT, PREC>()
#define TCALL(PREC) TCR(7, PREC), TCR(8, PREC), TCR(9, PREC), TCR(10, PREC), TCR(11, PREC), TCR(12, PREC), \
                    TCR(13, PREC), TC4(7, PREC), TC4(8, PREC)

extern const KernelEntry kTcF16Table[] = {TCALL(TC_FP16), TCALL(TC_FP16_SPLIT)};
extern const int kTcF16Count = sizeof(kTcF16Table) / sizeof(kTcF16Table[0]);

}  // namespace fftc

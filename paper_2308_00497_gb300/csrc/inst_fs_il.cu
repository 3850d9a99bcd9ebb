// Instantiations of the L2-resident four-step kernel, interleaved layout, n = 2^14 .. 2^20.
#include "fftc_fourstep_l2.cuh"

namespace fftc {

#define FS1(LOGM, E1, C1, LOGK, E2, C2) fs_entry<LOGM, E1, C1, LOGK, E2, C2, LAYOUT_IL>()

extern const FsEntry kFsIlTable[] = {
    FS1(7, 4, 16, 7, 4, 16),   // 2^14: 128 threads
    FS1(7, 4, 16, 8, 5, 16),   // 2^15: 128
    FS1(8, 4, 16, 8, 4, 16),   // 2^16: 256
    FS1(8, 4, 16, 9, 5, 16),   // 2^17: 256
    FS1(9, 5, 16, 9, 5, 16),   // 2^18: 256
    FS1(9, 5, 16, 10, 5, 8),   // 2^19: 256
    FS1(10, 5, 8, 10, 5, 8),   // 2^20: 256
};
extern const int kFsIlCount = sizeof(kFsIlTable) / sizeof(kFsIlTable[0]);

}  // namespace fftc

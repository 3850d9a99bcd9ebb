// Instantiation lists of the tensor-core passes (fftc_tc.cuh), one table per precision
// mode (inst_tc_*_m*.cu), 16 elements per thread (radix-16 stages) unless noted, both layouts:
//   single pass: n = 2^7, 2^8 as plain CTAs of 256 threads; n = 2^9 .. 2^14 as persistent
//                kernels fed by bulk copies (two landing buffers up to 2^12, one above),
//                one-buffer variants of 2^10 .. 2^12 (2^12 also with two lines a tile), and
//                32 elements per thread (radix-32 stages, one line a tile, one buffer) for
//                2^12 .. 2^14;
//   four-step:   n = 2^15 (M = 2^7, K = 2^8) and 2^16 (M = K = 2^8), 16 lines per tile;
//                pass 1 reads columns with plain loads or tensor-map boxes into one landing
//                buffer, pass 2 reads rows with plain loads or one bulk copy per tile into
//                two landing buffers and writes them transposed.
#pragma once

#include "fftc_pipe.cuh"

#define FFTC_TC_ROWS(M, LAY)                                                                                    \
    fftc::entry<7, 4, 32, fftc::KIND_ROWS, LAY, LAY, 0, M>(), fftc::entry<8, 4, 16, fftc::KIND_ROWS, LAY, LAY, 0, M>(), \
        fftc::pipe_entry<9, 4, 8, fftc::KIND_ROWS, LAY, LAY, 0, 2, true, M>(),                                   \
        fftc::pipe_entry<10, 4, 4, fftc::KIND_ROWS, LAY, LAY, 0, 2, true, M>(),                                  \
        fftc::pipe_entry<11, 4, 2, fftc::KIND_ROWS, LAY, LAY, 0, 2, true, M>(),                                  \
        fftc::pipe_entry<12, 4, 1, fftc::KIND_ROWS, LAY, LAY, 0, 2, true, M>(),                                  \
        fftc::pipe_entry<13, 4, 1, fftc::KIND_ROWS, LAY, LAY, 0, 1, true, M>(),                                  \
        fftc::pipe_entry<14, 4, 1, fftc::KIND_ROWS, LAY, LAY, 0, 1, true, M>(),                                  \
        fftc::pipe_entry<10, 4, 4, fftc::KIND_ROWS, LAY, LAY, 0, 1, true, M>(),                                  \
        fftc::pipe_entry<11, 4, 2, fftc::KIND_ROWS, LAY, LAY, 0, 1, true, M>(),                                  \
        fftc::pipe_entry<12, 4, 1, fftc::KIND_ROWS, LAY, LAY, 0, 1, true, M>(),                                  \
        fftc::pipe_entry<12, 4, 2, fftc::KIND_ROWS, LAY, LAY, 0, 1, true, M>(),                                  \
        fftc::pipe_entry<12, 5, 1, fftc::KIND_ROWS, LAY, LAY, 0, 1, true, M>(),                                  \
        fftc::pipe_entry<13, 5, 1, fftc::KIND_ROWS, LAY, LAY, 0, 1, true, M>(),                                  \
        fftc::pipe_entry<14, 5, 1, fftc::KIND_ROWS, LAY, LAY, 0, 1, true, M>()

#define FFTC_TC_COLS(M, LOGM, LOGK)                                                                   \
    fftc::entry<LOGM, 4, 16, fftc::KIND_COLS, fftc::LAYOUT_IL, fftc::LAYOUT_IL, LOGK, M>(),            \
        fftc::pipe_entry<LOGM, 4, 16, fftc::KIND_COLS, fftc::LAYOUT_IL, fftc::LAYOUT_IL, LOGK, 1, true, M>(), \
        fftc::pipe_entry<LOGM, 4, 16, fftc::KIND_COLS, fftc::LAYOUT_SPLIT, fftc::LAYOUT_IL, LOGK, 1, true, M>()
#define FFTC_TC_ROWST(M, LOGK, LOGM)                                                                      \
    fftc::entry<LOGK, 4, 16, fftc::KIND_ROWST, fftc::LAYOUT_IL, fftc::LAYOUT_IL, LOGM, M>(),              \
        fftc::entry<LOGK, 4, 16, fftc::KIND_ROWST, fftc::LAYOUT_IL, fftc::LAYOUT_SPLIT, LOGM, M>(),       \
        fftc::pipe_entry<LOGK, 4, 16, fftc::KIND_ROWST, fftc::LAYOUT_IL, fftc::LAYOUT_IL, LOGM, 2, true, M>(), \
        fftc::pipe_entry<LOGK, 4, 16, fftc::KIND_ROWST, fftc::LAYOUT_IL, fftc::LAYOUT_SPLIT, LOGM, 2, true, M>()
#define FFTC_TC_4STEP(M) \
    FFTC_TC_COLS(M, 7, 8), FFTC_TC_COLS(M, 8, 8), FFTC_TC_ROWST(M, 8, 7), FFTC_TC_ROWST(M, 8, 8)

// Instantiations of the pipelined persistent four-step passes (pass 1 fed by 2D tensor
// maps, pass 2 by one bulk copy per tile; fftc_pipe.cuh) for n = 2^14 .. 2^20 with
// compile-time strides, both layouts, and the host encoder of the pass-1 tensor maps.
#include <cstring>

#include "fftc_pipe.cuh"

namespace fftc {

#define PC2(LOGL, LOGE, C, LOGX, NBUF)                                          \
    pipe_entry<LOGL, LOGE, C, KIND_COLS, LAYOUT_IL, LAYOUT_IL, LOGX, NBUF>(),   \
        pipe_entry<LOGL, LOGE, C, KIND_COLS, LAYOUT_SPLIT, LAYOUT_IL, LOGX, NBUF>()
#define PT2(LOGL, LOGE, C, LOGX, NBUF)                                          \
    pipe_entry<LOGL, LOGE, C, KIND_ROWST, LAYOUT_IL, LAYOUT_IL, LOGX, NBUF>(),  \
        pipe_entry<LOGL, LOGE, C, KIND_ROWST, LAYOUT_IL, LAYOUT_SPLIT, LOGX, NBUF>()

extern const KernelEntry kPipe4Table[] = {
    PC2(7, 4, 16, 7, 2), PC2(7, 4, 16, 8, 2), PC2(8, 4, 16, 8, 2), PC2(8, 4, 16, 9, 2), PC2(10, 5, 8, 10, 2),
    PT2(7, 4, 16, 7, 2), PT2(8, 4, 16, 7, 2), PT2(8, 4, 16, 8, 2), PT2(9, 5, 8, 8, 2), PT2(10, 5, 8, 9, 2),
    PT2(10, 5, 8, 10, 2),
};
extern const int kPipe4Count = sizeof(kPipe4Table) / sizeof(kPipe4Table[0]);

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link)
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)f;
    }
    return fn;
}

// Pass-1 input as a 2D tensor: inner dimension the K columns of one row, outer the
// batch * M rows (row t of transform b is row b * M + t); box = C columns x min(M, 256) rows.
bool encode_cols_maps(const PassParams &p, int logl, int lines, int lay, CUtensorMap *tm) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t K = (cuuint64_t)p.in_elem, M = cuuint64_t(1) << logl;
    const cuuint64_t rows = (cuuint64_t)(p.total_lines >> p.log_lpt) * M;
    const cuuint32_t box[2] = {(cuuint32_t)lines, (cuuint32_t)(M < 256 ? M : 256)};
    const cuuint32_t estr[2] = {1, 1};
    const cuuint64_t dims[2] = {K, rows};
    if (lay == LAYOUT_IL) {
        const cuuint64_t strides[1] = {K * 8};
        return fn(&tm[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, (void *)p.in, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    const cuuint64_t strides[1] = {K * 4};
    if (fn(&tm[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)p.in, dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    return fn(&tm[1], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)(p.in + p.in_plane), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace fftc

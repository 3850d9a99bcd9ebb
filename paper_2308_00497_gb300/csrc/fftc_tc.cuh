// Radix-16 and radix-32 butterflies on the fifth-generation tensor cores (tcgen05, TMEM
// accumulators).
//
// A radix-R stage of Eq. 1 applies DFT_R to groups of R elements (the I (x) DFT_R factor;
// Table 1 FusedIKMV / FusedMKIV). On the tensor cores the R x R complex matrix
// W[t'][t] = w_R^(t' t) becomes one real product per group,
//     [yr | yi] = [xr | xi] . B,   B = [[ Wr^T, Wi^T], [-Wi^T, Wr^T]]   (2R x 2R),
// so 128 groups form one MMA of M = 128 rows (one group per row), K = 2R (R real and R
// imaginary inputs) and N = 2R (R real and R imaginary outputs), in 2R / 16 steps of K = 16.
// R = 16 is the radix-16 stage of 16-element threads; R = 32 the radix-32 stage of
// 32-element threads (one stage fewer, and one exchange fewer, for n = 2^10 .. 2^14). The
// dense product replaces the sparse radix-2 network of the CUDA-core path (the
// dense-versus-sparse contrast of Section 4).
//
// Operands are FP16 or BF16 with FP32 accumulation. In the split modes every operand is
// written as hi + lo (hi = rn(v), lo = rn(v - hi), the subtraction exact in FP32) and the
// three products hi.hi + lo.hi + hi.lo are accumulated into the same tensor-memory tile,
// which recovers most of the FP32 accuracy. FP16 data are scaled by 1/4 before each stage
// (exact) so that the growth of a stage stays far inside the FP16 range; the store scales
// back by 4 per stage. BF16 has FP32's exponent range.
//
// Data path of a group: the thread that owns the group in the CUDA-core pass kernel (R
// elements in registers, twiddled in FP32) writes its row of A into tensor memory with
// tcgen05.st (lane = row; warp w of the group owns lanes 32 (w mod 4) .. + 31), one thread
// of the 128-thread group issues the MMAs (A from tensor memory, B from shared memory) and
// commits them to an mbarrier, and every thread reads its row of D back from tensor
// memory (tcgen05.ld 32x32b) straight into the registers where the CUDA-core butterfly
// would have left it. The tile's shared memory is not touched, so the stage needs no CTA
// barrier of its own: the pass kernel goes on unchanged (FP32 twiddles, shared-memory
// exchange, coalesced HBM store).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fftc_device.cuh"
#include "fftc_internal.h"
#include "fftc_ptx.cuh"

namespace fftc {

// precision modes of the tensor-core passes (the fftc_precision values)
enum TcMode : int { TC_FP16 = 1, TC_BF16 = 2, TC_FP16_SPLIT = 3, TC_BF16_SPLIT = 4 };

__host__ __device__ constexpr bool tc_is_bf16(int mode) { return mode == TC_BF16 || mode == TC_BF16_SPLIT; }
__host__ __device__ constexpr bool tc_is_split(int mode) { return mode == TC_FP16_SPLIT || mode == TC_BF16_SPLIT; }

// Tensor-core area at the (128-byte aligned) start of dynamic shared memory, radix R:
//   [0, BB)         B hi: 2R rows n x 2R halves k, core-matrix layout (8-row groups R * 32 B apart)
//   [BB, 2 BB)      B lo (split modes)
//   [2 BB, + 64)    one mbarrier per 128-thread group (MMA completion)
//   [2 BB + 64]     TMEM base address written by tcgen05.alloc
__host__ __device__ constexpr int tc_b_bytes(int r) { return 2 * r * 2 * r * 2; }
__host__ __device__ constexpr int tc_area_bytes(int r) { return 2 * tc_b_bytes(r) + 128; }

__device__ __forceinline__ uint32_t tc_pack2(float a, float b, bool bf) {
    if (bf) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

__device__ __forceinline__ float2 tc_unpack2(uint32_t u, bool bf) {
    if (bf) return __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&u));
    return __half22float2(*reinterpret_cast<__half2 *>(&u));
}

// hi = rn(a, b); *lo = rn(a - hi.x, b - hi.y)
__device__ __forceinline__ uint32_t tc_split2(float a, float b, bool bf, uint32_t *lo) {
    const uint32_t hi = tc_pack2(a, b, bf);
    const float2 h = tc_unpack2(hi, bf);
    *lo = tc_pack2(a - h.x, b - h.y, bf);
    return hi;
}

__device__ __forceinline__ uint16_t tc_half_bits(float v, bool bf) {
    if (bf) {
        __nv_bfloat16 h = __float2bfloat16_rn(v);
        return *reinterpret_cast<uint16_t *>(&h);
    }
    __half h = __float2half_rn(v);
    return *reinterpret_cast<uint16_t *>(&h);
}

__device__ __forceinline__ float tc_half_value(uint16_t b, bool bf) {
    if (bf) return __bfloat162float(*reinterpret_cast<__nv_bfloat16 *>(&b));
    return __half2float(*reinterpret_cast<__half *>(&b));
}

// cos of 2 pi m / R (R | 64) from the quarter-period table of fftc_device.cuh
__device__ __forceinline__ float tc_cos(int m, int r) {
    const int a = (m * (64 / r)) & 63, q = a >> 4, f = a & 15;
    const float c = cos64_q(f), s = cos64_q(16 - f);
    return q == 0 ? c : (q == 1 ? -s : (q == 2 ? -c : s));
}
__device__ __forceinline__ float tc_sin(int m, int r) { return tc_cos(m - r / 4, r); }

// B[n][k] of the real form of DFT_R (forward, w_R = exp(-2 pi i / R)), n, k < 2R:
// yr_n = sum_t xr_t cos - xi_t (-sin), yi_n = sum_t xr_t (-sin) + xi_t cos, angle 2 pi n t / R
__device__ __forceinline__ float tc_b_value(int n, int k, int r) {
    const int m = (n % r) * (k % r);
    const float c = tc_cos(m, r), s = tc_sin(m, r);  // W = c - i s
    if (n < r) return k < r ? c : s;                 // Wr, -Wi
    return k < r ? -s : c;                           // Wi, Wr
}

// TMEM columns of a CTA of nt threads at radix r: 4r per 128-thread group (D tile and A
// rows), rounded up to a power of two (the allocation granule)
__host__ __device__ constexpr uint32_t tc_tmem_cols(int nt, int r) {
    const uint32_t c = (uint32_t)(nt / 128) * 4u * (uint32_t)r;
    return c <= 32u ? 32u : (c <= 64u ? 64u : (c <= 128u ? 128u : (c <= 256u ? 256u : 512u)));
}

template <int NT, int MODE, int R>
struct TcUnit {
    static_assert(R == 16 || R == 32, "radix 16 or 32");
    static_assert(NT % 128 == 0 && (NT / 128) * 4 * R <= 512, "whole 128-thread MMA groups within 512 TMEM columns");
    static_assert(MODE >= TC_FP16 && MODE <= TC_BF16_SPLIT, "a tensor-core precision mode");
    static constexpr bool BF = tc_is_bf16(MODE), SPLIT = tc_is_split(MODE);
    static constexpr int NWG = NT / 128;
    static constexpr int N2 = 2 * R;                    // N = K = 2R
    static constexpr int BB = tc_b_bytes(R);            // one B matrix
    static constexpr int BSBO = (N2 / 8) * 128;         // bytes between 8-row groups of B
    static constexpr int BARS = 2 * BB, TMEM_SLOT = 2 * BB + 64;
    // Tensor memory of 128-thread group g: GCOLS columns from GCOLS g, the FP32 D tile (2R
    // columns: R real then R imaginary outputs) then the A rows from column ACOL (FP16/BF16
    // pairs, the lower K in the low half: hi re, hi im, lo re, lo im, R / 2 columns each)
    static constexpr uint32_t GCOLS = 4 * R, ACOL = N2;
    static constexpr uint32_t COLS = tc_tmem_cols(NT, R);

    // every thread: DFT matrices into shared memory, mbarriers, TMEM columns
    __device__ static void setup(const PassParams &p, unsigned char *area) {
        (void)p;
        constexpr bool bf = BF;
        for (int i = threadIdx.x; i < N2 * N2; i += NT) {
            const int n = i / N2, k = i % N2;
            const float v = tc_b_value(n, k, R);
            const uint16_t hi = tc_half_bits(v, bf);
            const uint16_t lo = tc_half_bits(v - tc_half_value(hi, bf), bf);
            const int off = (n >> 3) * BSBO + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
            *reinterpret_cast<uint16_t *>(area + off) = hi;
            *reinterpret_cast<uint16_t *>(area + BB + off) = lo;
        }
        uint64_t *bars = reinterpret_cast<uint64_t *>(area + BARS);
        if (threadIdx.x == 0) {
            for (int g = 0; g < NWG; ++g) mbar_init(bars + g, 1);
            fence_mbar_init();
        }
        if (threadIdx.x < 32) tmem_alloc(reinterpret_cast<uint32_t *>(area + TMEM_SLOT), COLS);
        fence_proxy_async_smem();  // B is read by the tensor cores
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }

    __device__ static void teardown(unsigned char *area) {
        tc_fence_before();
        __syncthreads();
        if (threadIdx.x < 32) tmem_free(*reinterpret_cast<volatile uint32_t *>(area + TMEM_SLOT), COLS);
    }

    // v = DFT_R v for the thread's group (forward), on the tensor cores; `phase` is the
    // parity of this use of the group's mbarrier. Touches no shared memory but the DFT
    // matrices and the mbarrier, so the caller needs no barrier around it.
    __device__ __forceinline__ static void dft(const PassParams &p, float2 (&v)[R], unsigned char *area,
                                               uint32_t phase) {
        constexpr bool bf = BF, split = SPLIT;
        constexpr int H = R / 2;  // TMEM columns of one real part of a row (two halves each)
        const int tid = threadIdx.x, wg = tid >> 7, m = tid & 127;
        if constexpr (!bf) {
#pragma unroll
            for (int t = 0; t < R; ++t) {
                v[t].x *= 0.25f;
                v[t].y *= 0.25f;
            }
        }
        const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(area + TMEM_SLOT);
        const uint32_t gcol = tmem + GCOLS * wg;  // this group's columns, lane 0
        const uint32_t lanes = (uint32_t)(32 * ((tid >> 5) & 3)) << 16;  // this warp's lanes
        // A row: [hi re | hi im] then [lo re | lo im], R / 2 columns each part
        uint32_t hi[R], lo[split ? R : 1];
#pragma unroll
        for (int j = 0; j < H; ++j) {
            if constexpr (split) {
                hi[j] = tc_split2(v[2 * j].x, v[2 * j + 1].x, bf, &lo[j]);
                hi[H + j] = tc_split2(v[2 * j].y, v[2 * j + 1].y, bf, &lo[H + j]);
            } else {
                hi[j] = tc_pack2(v[2 * j].x, v[2 * j + 1].x, bf);
                hi[H + j] = tc_pack2(v[2 * j].y, v[2 * j + 1].y, bf);
            }
        }
        if constexpr (R == 16) {
            if constexpr (split) {
                uint32_t all[32];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    all[j] = hi[j];
                    all[16 + j] = lo[j];
                }
                tmem_st32(gcol + lanes + ACOL, all);
            } else {
                tmem_st16(gcol + lanes + ACOL, hi);
            }
        } else {
            tmem_st32(gcol + lanes + ACOL, hi);
            if constexpr (split) tmem_st32(gcol + lanes + ACOL + R, lo);
        }
        tmem_wait_st();
        tc_fence_before();
        named_bar(1 + wg, 128);  // every row of the group's A is in tensor memory
        uint64_t *bar = reinterpret_cast<uint64_t *>(area + BARS) + wg;
        if (m == 0) {
            tc_fence_after();
            const uint32_t idesc = umma_idesc_f16(bf, 128, N2);
            const uint32_t bhi = smem_u32(area), blo = bhi + BB, a = gcol + ACOL;
            // K = 16 steps over [re | im] of A (columns a + 8 i) against the matching 16 K rows
            // of B (two core-matrix chunks, 256 bytes apart)
#pragma unroll
            for (int i = 0; i < N2 / 16; ++i)
                umma_f16_ta(gcol, a + 8 * i, umma_desc(bhi + 256 * i, 128, BSBO), idesc, i > 0 ? 1u : 0u);
            if constexpr (split) {
#pragma unroll
                for (int i = 0; i < N2 / 16; ++i)  // lo.hi
                    umma_f16_ta(gcol, a + R + 8 * i, umma_desc(bhi + 256 * i, 128, BSBO), idesc, 1u);
#pragma unroll
                for (int i = 0; i < N2 / 16; ++i)  // hi.lo
                    umma_f16_ta(gcol, a + 8 * i, umma_desc(blo + 256 * i, 128, BSBO), idesc, 1u);
            }
            umma_commit(bar);
        }
        const long long limit = p.spin_limit > 0 ? (long long)p.spin_limit : kMbarSpinLimit;
        if (!mbar_wait_sleepy(bar, phase, limit) && m == 0 && p.err) atomicExch(p.err, 3);
        tc_fence_after();
        __syncwarp();  // tcgen05.ld is warp-collective
        // D row: R real outputs in columns 0 .. R - 1, then R imaginary outputs
        if constexpr (R == 16) {
            uint32_t r[32];
            tmem_ld32(gcol + lanes, r);
            tmem_wait_ld();
#pragma unroll
            for (int t = 0; t < 16; ++t) v[t] = make_float2(__uint_as_float(r[t]), __uint_as_float(r[16 + t]));
        } else {
            uint32_t r[32], q[32];
            tmem_ld32(gcol + lanes, r);
            tmem_ld32(gcol + lanes + R, q);
            tmem_wait_ld();
#pragma unroll
            for (int t = 0; t < 32; ++t) v[t] = make_float2(__uint_as_float(r[t]), __uint_as_float(q[t]));
        }
        tc_fence_before();
    }
};

}  // namespace fftc

// Radix-16 butterflies on the fifth-generation tensor cores (tcgen05, TMEM accumulators).
//
// A radix-16 stage of Eq. 1 applies DFT_16 to groups of 16 elements (the I (x) DFT_R
// factor; Table 1 FusedIKMV / FusedMKIV). On the tensor cores the 16 x 16 complex matrix
// W16[t'][t] = w_16^(t' t) becomes one real product per group,
//     [yr | yi] = [xr | xi] . B,   B = [[ Wr^T, Wi^T], [-Wi^T, Wr^T]]   (32 x 32),
// so 128 groups form one MMA of M = 128 rows (one group per row), K = 32 (16 real and 16
// imaginary inputs) and N = 32 (16 real and 16 imaginary outputs), in two K = 16 steps.
// The dense product replaces the sparse radix-2 network of the CUDA-core path (the
// dense-versus-sparse contrast of Section 4).
//
// Operands are FP16 or BF16 with FP32 accumulation. In the split modes every operand is
// written as hi + lo (hi = rn(v), lo = rn(v - hi), the subtraction exact in FP32) and the
// three products hi.hi + lo.hi + hi.lo are accumulated into the same tensor-memory tile
// (six K = 16 steps), which recovers most of the FP32 accuracy. FP16 data are scaled by
// 1/4 before each stage (exact) so that the growth of a radix-16 stage cannot leave the
// FP16 range; the store scales back by 4 per stage. BF16 has FP32's exponent range.
//
// Data path of a group: the thread that owns the group in the CUDA-core pass kernel (16
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

// Tensor-core area at the (128-byte aligned) start of dynamic shared memory:
//   [0, 2048)     B hi: 32 rows n x 32 halves k, core-matrix layout (row group 512 B apart)
//   [2048, 4096)  B lo (split modes)
//   [4096, 4160)  one mbarrier per 128-thread group (MMA completion)
//   [4160]        TMEM base address written by tcgen05.alloc
constexpr int kTcAreaBytes = 4096 + 128;
constexpr int kTcBLo = 2048, kTcBars = 4096, kTcTmem = 4096 + 64;
// Tensor memory of a 128-thread group g: 64 columns from 64 g, the FP32 D tile (32 columns:
// 16 real then 16 imaginary outputs) then the A rows (FP16/BF16 pairs, lower K in the low
// half: hi re, hi im, lo re, lo im, 8 columns each = K 0..15 of each part)
constexpr uint32_t kTcGroupCols = 64, kTcACol = 32;

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

// cos and sin of 2 pi m / 16 from the quarter-period table of fftc_device.cuh
__device__ __forceinline__ float tc_cos16(int m) {
    m &= 15;
    const int q = m >> 2, r = m & 3;
    const float c = cos64_q(4 * r), s = cos64_q(16 - 4 * r);
    return q == 0 ? c : (q == 1 ? -s : (q == 2 ? -c : s));
}
__device__ __forceinline__ float tc_sin16(int m) { return tc_cos16(m - 4); }

// B[n][k] of the real form of DFT_16 (forward, w_16 = exp(-2 pi i / 16)):
// yr_n = sum_t xr_t cos - xi_t (-sin), yi_n = sum_t xr_t (-sin) + xi_t cos, angle 2 pi n t / 16
__device__ __forceinline__ float tc_b_value(int n, int k) {
    const int no = n & 15, t = k & 15, m = no * t;
    const float c = tc_cos16(m), s = tc_sin16(m);  // W = c - i s
    if (n < 16) return k < 16 ? c : s;             // Wr, -Wi
    return k < 16 ? -s : c;                        // Wi, Wr
}

// TMEM columns of a CTA of nt threads: 64 per 128-thread group (D tile and A rows), a power
// of two (the allocation granule)
__host__ __device__ constexpr uint32_t tc_tmem_cols(int nt) {
    return nt <= 128 ? 64u : (nt <= 256 ? 128u : (nt <= 512 ? 256u : 512u));
}

template <int NT, int MODE>
struct TcUnit {
    static_assert(NT % 128 == 0 && NT <= 1024, "whole 128-thread MMA groups");
    static_assert(MODE >= TC_FP16 && MODE <= TC_BF16_SPLIT, "a tensor-core precision mode");
    static constexpr bool BF = tc_is_bf16(MODE), SPLIT = tc_is_split(MODE);
    static constexpr int NWG = NT / 128;
    static constexpr uint32_t COLS = tc_tmem_cols(NT);

    // every thread: DFT matrices into shared memory, mbarriers, TMEM columns
    __device__ static void setup(const PassParams &p, unsigned char *area) {
        (void)p;
        constexpr bool bf = BF;
        for (int i = threadIdx.x; i < 32 * 32; i += NT) {
            const int n = i >> 5, k = i & 31;
            const float v = tc_b_value(n, k);
            const uint16_t hi = tc_half_bits(v, bf);
            const uint16_t lo = tc_half_bits(v - tc_half_value(hi, bf), bf);
            const int off = (n >> 3) * 512 + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
            *reinterpret_cast<uint16_t *>(area + off) = hi;
            *reinterpret_cast<uint16_t *>(area + kTcBLo + off) = lo;
        }
        uint64_t *bars = reinterpret_cast<uint64_t *>(area + kTcBars);
        if (threadIdx.x == 0) {
            for (int g = 0; g < NWG; ++g) mbar_init(bars + g, 1);
            fence_mbar_init();
        }
        if (threadIdx.x < 32) tmem_alloc(reinterpret_cast<uint32_t *>(area + kTcTmem), COLS);
        fence_proxy_async_smem();  // B is read by the tensor cores
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }

    __device__ static void teardown(unsigned char *area) {
        tc_fence_before();
        __syncthreads();
        if (threadIdx.x < 32) tmem_free(*reinterpret_cast<volatile uint32_t *>(area + kTcTmem), COLS);
    }

    // v = DFT_16 v for the thread's group (forward), on the tensor cores; `phase` is the
    // parity of this use of the group's mbarrier. Touches no shared memory but the DFT
    // matrices and the mbarrier, so the caller needs no barrier around it.
    __device__ __forceinline__ static void dft16(const PassParams &p, float2 (&v)[16], unsigned char *area,
                                                 uint32_t phase) {
        constexpr bool bf = BF, split = SPLIT;
        const int tid = threadIdx.x, wg = tid >> 7, m = tid & 127;
        if constexpr (!bf) {
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                v[t].x *= 0.25f;
                v[t].y *= 0.25f;
            }
        }
        const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(area + kTcTmem);
        const uint32_t gcol = tmem + kTcGroupCols * wg;  // this group's columns, lane 0
        const uint32_t lanes = (uint32_t)(32 * ((tid >> 5) & 3)) << 16;  // this warp's lanes
        if constexpr (split) {
            uint32_t r[32];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                r[j] = tc_split2(v[2 * j].x, v[2 * j + 1].x, bf, &r[16 + j]);
                r[8 + j] = tc_split2(v[2 * j].y, v[2 * j + 1].y, bf, &r[24 + j]);
            }
            tmem_st32(gcol + lanes + kTcACol, r);
        } else {
            uint32_t r[16];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                r[j] = tc_pack2(v[2 * j].x, v[2 * j + 1].x, bf);
                r[8 + j] = tc_pack2(v[2 * j].y, v[2 * j + 1].y, bf);
            }
            tmem_st16(gcol + lanes + kTcACol, r);
        }
        tc_fence_before();
        named_bar(1 + wg, 128);  // every row of the group's A is in tensor memory
        uint64_t *bar = reinterpret_cast<uint64_t *>(area + kTcBars) + wg;
        if (m == 0) {
            tc_fence_after();
            const uint32_t idesc = umma_idesc_f16(bf, 128, 32);
            const uint32_t bhi = smem_u32(area), blo = bhi + kTcBLo, a = gcol + kTcACol;
            // K = 16 steps: (A columns, B chunks) = (re, re-rows of B), (im, im-rows of B)
            umma_f16_ta(gcol, a, umma_desc(bhi, 128, 512), idesc, 0);
            umma_f16_ta(gcol, a + 8, umma_desc(bhi + 256, 128, 512), idesc, 1);
            if constexpr (split) {
                umma_f16_ta(gcol, a + 16, umma_desc(bhi, 128, 512), idesc, 1);  // lo.hi
                umma_f16_ta(gcol, a + 24, umma_desc(bhi + 256, 128, 512), idesc, 1);
                umma_f16_ta(gcol, a, umma_desc(blo, 128, 512), idesc, 1);  // hi.lo
                umma_f16_ta(gcol, a + 8, umma_desc(blo + 256, 128, 512), idesc, 1);
            }
            umma_commit(bar);
        }
        const long long limit = p.spin_limit > 0 ? (long long)p.spin_limit : kMbarSpinLimit;
        if (!mbar_wait_sleepy(bar, phase, limit) && m == 0 && p.err) atomicExch(p.err, 3);
        tc_fence_after();
        __syncwarp();  // tcgen05.ld is warp-collective
        uint32_t r[32];
        tmem_ld32(gcol + lanes, r);
#pragma unroll
        for (int t = 0; t < 16; ++t) v[t] = make_float2(__uint_as_float(r[t]), __uint_as_float(r[16 + t]));
        tc_fence_before();
    }
};

}  // namespace fftc

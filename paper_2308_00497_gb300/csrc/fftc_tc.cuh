// Tensor-core radix-16 Stockham pass.
//
// Every radix-16 stage computes Y = W16 X for groups of 16 inputs, W16[t'][t] =
// w_16^(t' t), as the real block product
//     [Yr]   [Wr  -Wi] [Xr]
//     [Yi] = [Wi   Wr] [Xi]
// on the tensor cores: mma.sync m16n8k16 with FP16 or BF16 operands and FP32
// accumulation, one MMA tile = 16 outputs x 8 butterflies. The twiddles of Eq. 1
// (the diagonal D between stages) stay FP32 on the CUDA cores and are applied before
// the operands are rounded. In the split modes every operand is written as hi + lo
// (hi = rn(v), lo = rn(v - hi)) and the three products hi*hi + hi*lo + lo*hi are
// accumulated, which recovers most of the FP32 accuracy. A leftover radix-2/4/8
// stage (log2 L not a multiple of 4) runs in FP32 first.
//
// Data path of a CTA (C lines of length L): HBM -> shared (coalesced), every stage
// shared -> registers -> tensor cores -> shared (two buffers), shared -> HBM.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fftc_device.cuh"
#include "fftc_internal.h"

namespace fftc {

enum TcPrec : int { TC_FP16 = 1, TC_BF16 = 2, TC_FP16_SPLIT = 3, TC_BF16_SPLIT = 4 };

template <int PREC>
struct TcOps {
    static constexpr bool BF = (PREC == TC_BF16 || PREC == TC_BF16_SPLIT);
    static constexpr bool SPLIT = (PREC == TC_FP16_SPLIT || PREC == TC_BF16_SPLIT);
    // FP16 operands are scaled by 1/4 per stage (exact) to keep the growth of a
    // radix-16 stage inside the FP16 range; BF16 has the FP32 exponent range.
    static constexpr float IN_SCALE = BF ? 1.0f : 0.25f;
    static constexpr float OUT_SCALE = BF ? 1.0f : 4.0f;

    // pack (a, b) -> .b32 with a in the low half; *lo gets the packed remainders
    __device__ __forceinline__ static uint32_t pack(float a, float b, uint32_t *lo) {
        if constexpr (BF) {
            __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
            if (lo) {
                float2 hf = __bfloat1622float2(h);
                __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
                *lo = *reinterpret_cast<uint32_t *>(&l);
            }
            return *reinterpret_cast<uint32_t *>(&h);
        } else {
            __half2 h = __floats2half2_rn(a, b);
            if (lo) {
                float2 hf = __half22float2(h);
                __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
                *lo = *reinterpret_cast<uint32_t *>(&l);
            }
            return *reinterpret_cast<uint32_t *>(&h);
        }
    }

    __device__ __forceinline__ static void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
        if constexpr (BF) {
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};\n"
                : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
        } else {
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};\n"
                : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
        }
    }
};

// cos and sin of 2*pi*m/16
__device__ __forceinline__ float cos16(int m) {
    m &= 15;
    const int q = m >> 2, r = m & 3;
    const float c = cos64_q(4 * r), s = cos64_q(16 - 4 * r);
    return q == 0 ? c : (q == 1 ? -s : (q == 2 ? -c : s));
}
__device__ __forceinline__ float sin16(int m) { return cos16(m - 4); }

template <int LOGL, int C, int KIND, int LIN, int LOUT, int PREC>
struct TcPass {
    using Sc = Sched<LOGL, 4, true>;  // leftover radix first, then radix-16 stages
    using Ops = TcOps<PREC>;
    static constexpr int L = 1 << LOGL, S = Sc::S, NT = 256, NW = NT / 32;
    static constexpr int ROW = L / 16;            // one row per input index t of a radix-16 stage
    static constexpr int PITCH = L + 33;          // rows padded by 2 words, lines by one more (odd)
    static constexpr int SMEM = 2 * C * PITCH * (int)sizeof(float2);
    static_assert(LOGL >= 7, "an MMA tile needs 8 butterflies of one line");
    static_assert((C * L) % 128 == 0, "whole MMA tiles");

    __device__ __forceinline__ static int rp(int a) { return (a / ROW) * (ROW + 2) + (a % ROW); }

    __device__ __forceinline__ static int64_t line_base(const PassParams &p, int64_t g, int64_t tr, int64_t line) {
        return (g >> p.log_lpt) * tr + (g & ((int64_t(1) << p.log_lpt) - 1)) * line;
    }

    // Element (c, a) of the tile handled by iteration `it` of thread `tid`. Row-contiguous
    // kinds walk a line with consecutive threads; the column kind walks C lines.
    static constexpr int ITER = C * L / NT;
    static_assert(ITER * NT == C * L, "whole tiles per thread");
    template <bool TAU>
    __device__ __forceinline__ static void coord(int tid, int it, int &c, int &a) {
        const int i = tid + it * NT;
        if constexpr (TAU) {
            c = i >> LOGL;
            a = i & (L - 1);
        } else {
            c = i % C;
            a = i / C;
        }
    }

    // HBM -> shared, all loads of a thread issued before its first store
    __device__ static void copy_in(const PassParams &p, float2 *buf, int64_t g0) {
        constexpr bool TAU = (KIND != KIND_COLS);
        constexpr int CH = ITER < 16 ? ITER : 16;  // loads in flight per thread
        const int es = (int)p.in_elem;
#pragma unroll
        for (int b0 = 0; b0 < ITER; b0 += CH) {
            float2 x[CH];
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                int c, a;
                coord<TAU>(threadIdx.x, b0 + u, c, a);
                const int64_t g = g0 + c;
                x[u] = make_float2(0.f, 0.f);
                if (g < p.total_lines) {
                    const int64_t off = line_base(p, g, p.in_tr, p.in_line) + (int64_t)a * es;
                    if constexpr (LIN == LAYOUT_IL) {
                        if constexpr (KIND == KIND_ROWST) x[u] = __ldcg(reinterpret_cast<const float2 *>(p.in) + off);
                        else x[u] = __ldcs(reinterpret_cast<const float2 *>(p.in) + off);
                    } else {
                        x[u].x = __ldcs(p.in + off);
                        x[u].y = __ldcs(p.in + p.in_plane + off);
                    }
                    if (p.conj_in) x[u].y = -x[u].y;
                }
            }
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                int c, a;
                coord<TAU>(threadIdx.x, b0 + u, c, a);
                buf[c * PITCH + rp(a)] = x[u];
            }
        }
    }

    // shared -> HBM (with the inter-pass twiddle for the column kind)
    __device__ static void copy_out(const PassParams &p, const float2 *buf, int64_t g0) {
        constexpr bool TAU = (KIND == KIND_ROWS);
        const int es = (int)p.out_elem;
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            int c, a;
            coord<TAU>(threadIdx.x, it, c, a);
            const int64_t g = g0 + c;
            if (g >= p.total_lines) continue;
            float2 x = buf[c * PITCH + rp(a)];
            const int l = (int)(g & ((int64_t(1) << p.log_lpt) - 1));
            if constexpr (KIND == KIND_COLS) {
                if (p.tw2_full) {
                    x = cmul(x, __ldg(p.tw2_full + l * (int)p.out_line + a * es));
                } else {
                    const int m = (l * a) & ((1 << p.log_n2) - 1);
                    x = cmul(x, cmul(__ldg(p.tw2_lo + (m & ((1 << p.tw2_lo_bits) - 1))),
                                     __ldg(p.tw2_hi + (m >> p.tw2_lo_bits))));
                }
            }
            if (p.conj_out) x.y = -x.y;
            const int64_t off = line_base(p, g, p.out_tr, p.out_line) + (int64_t)a * es;
            if constexpr (KIND == KIND_COLS) {
                __stcg(reinterpret_cast<float2 *>(p.out) + off, x);
            } else if constexpr (LOUT == LAYOUT_IL) {
                __stcs(reinterpret_cast<float2 *>(p.out) + off, x);
            } else {
                __stcs(p.out + off, x.x);
                __stcs(p.out + p.out_plane + off, x.y);
            }
        }
    }

    // FP32 leftover stage (first stage, Ns = 1, radix R < 16)
    template <int R>
    __device__ static void small_stage(const float2 *src, float2 *dst) {
        for (int i = threadIdx.x; i < C * (L / R); i += NT) {
            const int c = i / (L / R), j = i % (L / R);
            float2 v[R];
#pragma unroll
            for (int t = 0; t < R; ++t) v[t] = src[c * PITCH + rp(j + t * (L / R))];
            dft<R>(v);
#pragma unroll
            for (int t = 0; t < R; ++t) dst[c * PITCH + rp(j * R + t)] = v[t];
        }
    }

    // one radix-16 stage on the tensor cores
    template <int LNS>
    __device__ static void tc_stage(const PassParams &p, const float2 *src, float2 *dst, const uint32_t (&wr)[4],
                                    const uint32_t (&wi)[4], const uint32_t (&nwi)[4], const uint32_t (&wrl)[4],
                                    const uint32_t (&wil)[4], const uint32_t (&nwil)[4], const float2 *tw) {
        constexpr int NS = 1 << LNS;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int g = lane >> 2, tig = lane & 3;
        const int tt[4] = {2 * tig, 2 * tig + 1, 2 * tig + 8, 2 * tig + 9};
        constexpr int GROUPS = C * L / 128;
        for (int grp = warp; grp < GROUPS; grp += NW) {
            const int c = grp / (L / 128), j0 = (grp % (L / 128)) * 8;
            const float2 *s = src + c * PITCH;
            const int j = j0 + g;
            float2 x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = s[j + tt[u] * (ROW + 2)];  // = rp(j + t ROW), j < ROW
            if constexpr (NS > 1) {
                const int k = j & (NS - 1);
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (tt[u] > 0) x[u] = cmul(x[u], __ldg(tw + (tt[u] - 1) * NS + k));
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                x[u].x *= Ops::IN_SCALE;
                x[u].y *= Ops::IN_SCALE;
            }
            uint32_t brl[2], bil[2];
            const uint32_t br0 = Ops::pack(x[0].x, x[1].x, Ops::SPLIT ? &brl[0] : nullptr);
            const uint32_t br1 = Ops::pack(x[2].x, x[3].x, Ops::SPLIT ? &brl[1] : nullptr);
            const uint32_t bi0 = Ops::pack(x[0].y, x[1].y, Ops::SPLIT ? &bil[0] : nullptr);
            const uint32_t bi1 = Ops::pack(x[2].y, x[3].y, Ops::SPLIT ? &bil[1] : nullptr);
            float yr[4] = {0.f, 0.f, 0.f, 0.f}, yi[4] = {0.f, 0.f, 0.f, 0.f};
            Ops::mma(yr, wr, br0, br1);    // Wr Xr
            Ops::mma(yr, nwi, bi0, bi1);   // - Wi Xi
            Ops::mma(yi, wi, br0, br1);    // Wi Xr
            Ops::mma(yi, wr, bi0, bi1);    // Wr Xi
            if constexpr (Ops::SPLIT) {
                Ops::mma(yr, wr, brl[0], brl[1]);
                Ops::mma(yr, nwi, bil[0], bil[1]);
                Ops::mma(yi, wi, brl[0], brl[1]);
                Ops::mma(yi, wr, bil[0], bil[1]);
                Ops::mma(yr, wrl, br0, br1);
                Ops::mma(yr, nwil, bi0, bi1);
                Ops::mma(yi, wil, br0, br1);
                Ops::mma(yi, wrl, bi0, bi1);
            }
            // d[0]: (t' = g, butterfly 2 tig), d[1]: (g, 2 tig + 1), d[2]: (g + 8, 2 tig), d[3]: (g + 8, 2 tig + 1)
            float2 *d = dst + c * PITCH;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int jj = j0 + 2 * tig + (r & 1);
                const int tp = g + ((r & 2) ? 8 : 0);
                const int pos = ((jj >> LNS) << (LNS + 4)) + (jj & (NS - 1)) + tp * NS;
                d[rp(pos)] = make_float2(yr[r] * Ops::OUT_SCALE, yi[r] * Ops::OUT_SCALE);
            }
        }
    }

    template <int s>
    __device__ static void stages(const PassParams &p, float2 *a, float2 *b, const uint32_t (&wr)[4],
                                  const uint32_t (&wi)[4], const uint32_t (&nwi)[4], const uint32_t (&wrl)[4],
                                  const uint32_t (&wil)[4], const uint32_t (&nwil)[4]) {
        constexpr int LR = Sc::lr(s), LNS = Sc::lns(s);
        if constexpr (LR < 4) {
            small_stage<1 << LR>(a, b);
        } else {
            tc_stage<LNS>(p, a, b, wr, wi, nwi, wrl, wil, nwil, p.tw + Sc::tw_off(s));
        }
        __syncthreads();
        if constexpr (s + 1 < S) stages<s + 1>(p, b, a, wr, wi, nwi, wrl, wil, nwil);
    }

    __device__ static void run(const PassParams &p) {
        extern __shared__ float2 sm_tc[];
        float2 *a = sm_tc, *b = sm_tc + C * PITCH;
        // W16 fragments (A operand, rows t' = g, g + 8; columns t = 2 tig (+1), 2 tig + 8 (+9))
        const int lane = threadIdx.x & 31, g = lane >> 2, tig = lane & 3;
        uint32_t wr[4], wi[4], nwi[4], wrl[4] = {0, 0, 0, 0}, wil[4] = {0, 0, 0, 0}, nwil[4] = {0, 0, 0, 0};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int row = g + ((r & 1) ? 8 : 0), col = 2 * tig + ((r & 2) ? 8 : 0);
            const int m0 = (row * col) & 15, m1 = (row * (col + 1)) & 15;
            // W = cos - i sin (forward): Wr = cos, Wi = -sin
            wr[r] = Ops::pack(cos16(m0), cos16(m1), Ops::SPLIT ? &wrl[r] : nullptr);
            wi[r] = Ops::pack(-sin16(m0), -sin16(m1), Ops::SPLIT ? &wil[r] : nullptr);
            nwi[r] = Ops::pack(sin16(m0), sin16(m1), Ops::SPLIT ? &nwil[r] : nullptr);
        }
        const int64_t g0 = (int64_t)blockIdx.x * C;
        copy_in(p, a, g0);
        __syncthreads();
        stages<0>(p, a, b, wr, wi, nwi, wrl, wil, nwil);
        copy_out(p, (S % 2) ? b : a, g0);
    }
};

template <int LOGL, int C, int KIND, int LIN, int LOUT, int PREC>
__global__ void __launch_bounds__(256) k_tc(const __grid_constant__ PassParams p) {
    TcPass<LOGL, C, KIND, LIN, LOUT, PREC>::run(p);
}

template <int LOGL, int C, int KIND, int LIN, int LOUT, int PREC>
cudaError_t launch_tc(const PassParams &p, cudaStream_t st) {
    using P = TcPass<LOGL, C, KIND, LIN, LOUT, PREC>;
    const int64_t blocks = (p.total_lines + C - 1) / C;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
    k_tc<LOGL, C, KIND, LIN, LOUT, PREC><<<(unsigned)blocks, P::NT, P::SMEM, st>>>(p);
    return cudaGetLastError();
}

template <int LOGL, int C, int KIND, int LIN, int LOUT, int PREC>
cudaError_t prepare_tc() {
    using P = TcPass<LOGL, C, KIND, LIN, LOUT, PREC>;
    if (P::SMEM <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(k_tc<LOGL, C, KIND, LIN, LOUT, PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                P::SMEM);
}

template <int LOGL, int C, int KIND, int LIN, int LOUT, int PREC>
constexpr KernelEntry tc_entry() {
    using P = TcPass<LOGL, C, KIND, LIN, LOUT, PREC>;
    return KernelEntry{KIND,   LOGL,   4, C, LIN, LOUT, P::NT, P::SMEM, &launch_tc<LOGL, C, KIND, LIN, LOUT, PREC>,
                       &prepare_tc<LOGL, C, KIND, LIN, LOUT, PREC>, PREC, 0, 0};
}

}  // namespace fftc

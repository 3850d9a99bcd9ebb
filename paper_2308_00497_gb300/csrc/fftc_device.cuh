// Device building blocks of the fused Stockham kernels: complex arithmetic, the
// in-register radix-R DFT, the radix schedule of a line and the shared-memory
// swizzle of each exchange.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fftc {

// ---------------------------------------------------------------------------
// complex helpers (float2 = re, im)
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// ask L2 to fetch the line holding `p` (no register result, no fault semantics needed:
// callers pass addresses inside their buffers)
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// cos(2*pi*m/64) for m = 0..16 (a quarter period): cos(pi*m/32).
__host__ __device__ __forceinline__ float cos64_q(int m) {
    switch (m) {
        case 0: return 1.0f;
        case 1: return 0.99518472667219693f;
        case 2: return 0.98078528040323043f;
        case 3: return 0.95694033573220882f;
        case 4: return 0.92387953251128674f;
        case 5: return 0.88192126434835505f;
        case 6: return 0.83146961230254524f;
        case 7: return 0.77301045336273699f;
        case 8: return 0.70710678118654757f;
        case 9: return 0.63439328416364549f;
        case 10: return 0.55557023301960229f;
        case 11: return 0.47139673682599781f;
        case 12: return 0.38268343236508984f;
        case 13: return 0.29028467725446233f;
        case 14: return 0.19509032201612833f;
        case 15: return 0.09801714032956077f;
        default: return 0.0f;
    }
}

// x * w_64^m with w_64 = exp(-2*pi*i/64); m is a compile-time constant after
// unrolling, so the branches fold and the trivial factors (1, -i, -1, +i and the
// sqrt(1/2) pair) cost no multiplies.
__host__ __device__ __forceinline__ float2 mul_w64(float2 x, int m) {
    m &= 63;
    if (m == 0) return x;
    if (m == 16) return make_float2(x.y, -x.x);   // * (-i)
    if (m == 32) return make_float2(-x.x, -x.y);  // * (-1)
    if (m == 48) return make_float2(-x.y, x.x);   // * (+i)
    if (m == 8 || m == 24 || m == 40 || m == 56) {
        const float h = 0.70710678118654757f;
        float2 y;
        if (m == 8) y = make_float2(x.x + x.y, x.y - x.x);         // (1 - i)/sqrt2
        else if (m == 24) y = make_float2(x.y - x.x, -x.x - x.y);  // (-1 - i)/sqrt2
        else if (m == 40) y = make_float2(-x.x - x.y, x.x - x.y);  // (-1 + i)/sqrt2
        else y = make_float2(x.x - x.y, x.x + x.y);                // (1 + i)/sqrt2
        return make_float2(y.x * h, y.y * h);
    }
    // general: w = cos(t) - i sin(t), t = 2*pi*m/64
    int q = m >> 4, r = m & 15;
    float c, s;  // cos(t), sin(t)
    if (q == 0) { c = cos64_q(r); s = cos64_q(16 - r); }
    else if (q == 1) { c = -cos64_q(16 - r); s = cos64_q(r); }
    else if (q == 2) { c = -cos64_q(r); s = -cos64_q(16 - r); }
    else { c = cos64_q(16 - r); s = -cos64_q(r); }
    return make_float2(x.x * c + x.y * s, x.y * c - x.x * s);
}

__host__ __device__ constexpr int bitrev(int v, int bits) {
    int r = 0;
    for (int i = 0; i < bits; ++i) r |= ((v >> i) & 1) << (bits - 1 - i);
    return r;
}

__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v >> 1); }

// Forward DFT_R (R = 2..64) of a[0..R) in registers, result in natural order:
// a radix-2 decimation-in-frequency network with constant twiddles, followed by
// a compile-time bit-reversal renaming of the registers.
template <int R>
__host__ __device__ __forceinline__ void dft(float2 *a) {
    static_assert(R >= 1 && R <= 64 && (R & (R - 1)) == 0, "radix must be a power of two <= 64");
    if constexpr (R > 1) {
#pragma unroll
        for (int span = R / 2; span >= 1; span >>= 1) {
#pragma unroll
            for (int g = 0; g < R; g += 2 * span) {
#pragma unroll
                for (int k = 0; k < span; ++k) {
                    float2 x = a[g + k], y = a[g + k + span];
                    a[g + k] = cadd(x, y);
                    a[g + k + span] = mul_w64(csub(x, y), k * (64 / (2 * span)));
                }
            }
        }
        float2 b[R];
#pragma unroll
        for (int f = 0; f < R; ++f) b[f] = a[bitrev(f, ilog2(R))];
#pragma unroll
        for (int f = 0; f < R; ++f) a[f] = b[f];
    }
}

// ---------------------------------------------------------------------------
// Radix schedule of one line of length L = 2^LOGL with E = 2^LOGE elements per
// thread: S stages of radix E, except that when LOGE does not divide LOGL the last
// stage takes the remainder radix 2^(LOGL mod LOGE).
// Stage s has sub-transform length Ns = product of the earlier radices (the
// Stockham "Ns"). Per-stage twiddle tables (stage s >= 1) hold w_{Ns R}^{t k} at
// [(t-1) Ns + k], t = 1..R-1, k < Ns, concatenated in stage order.
// ---------------------------------------------------------------------------
template <int LOGL, int LOGE>
struct Sched {
    static_assert(LOGE >= 1 && LOGE <= LOGL, "need 2 <= E <= L");
    static constexpr int L = 1 << LOGL;
    static constexpr int E = 1 << LOGE;
    static constexpr int TPL = L / E;  // threads per line
    static constexpr int S = (LOGL + LOGE - 1) / LOGE;
    static constexpr int REM = LOGL % LOGE;
    __host__ __device__ static constexpr int lr(int s) {
        return (REM && s == S - 1) ? REM : LOGE;
    }
    __host__ __device__ static constexpr int lns(int s) {
        int acc = 0;
        for (int i = 0; i < s; ++i) acc += lr(i);
        return acc;
    }
    __host__ __device__ static constexpr int tw_off(int s) {
        int o = 0;
        for (int i = 1; i < s; ++i) o += ((1 << lr(i)) - 1) << lns(i);
        return o;
    }
    static constexpr int tw_total = tw_off(S);
};

}  // namespace fftc

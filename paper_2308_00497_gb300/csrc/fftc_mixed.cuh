// Runtime-radix Stockham pass: FP32 for n = 2^a 3^b 5^c 7^d that are not powers of two,
// FP64 (complex128) for every supported n. The element type V is float2 or double2.
//
// One CTA transforms C lines of length L held in shared memory. The radices r_s of the
// line (from {16, 15, 14, 12, 10, 9, 8, 7, 6, 5, 4, 3, 2}, product L) are runtime values,
// so one kernel serves
// every length; each stage s (Ns = r_0 ... r_{s-1}) applies one factor of Eq. 1 to every
// butterfly group of every line:
//   read    a[t] = x[j + t L/r]                       (the stride permutation)
//   twiddle a[t] *= w_{Ns r}^{t (j mod Ns)}            (the diagonal, FP64-built table)
//   DFT_r   in registers (radix-2 networks for powers of two, paired sums for 3, 5, 7,
//           and Eq. 1 once more with compile-time twiddles for composite r)
//   write   y[(j / Ns) Ns r + (j mod Ns) + t Ns] = a[t] (autosort)
// between two shared buffers (ping-pong, one barrier per stage). The tile moves through
// HBM once: a coalesced load into shared memory, the stages, a coalesced store; the
// four-step kinds are the same as the power-of-two passes (columns at stride K times the
// inter-pass diagonal w_N^(b t'), or rows stored transposed), with lines addressed by
// division by invariant integers instead of shifts.
#pragma once

#include <type_traits>

#include "fftc_ctrig.h"
#include "fftc_device.cuh"
#include "fftc_internal.h"

namespace fftc {

constexpr int kMixedMaxStages = 24;

template <typename V>
struct CplxT;
template <>
struct CplxT<float2> {
    using S = float;
    __host__ __device__ static float2 make(float x, float y) { return make_float2(x, y); }
};
template <>
struct CplxT<double2> {
    using S = double;
    __host__ __device__ static double2 make(double x, double y) { return make_double2(x, y); }
};
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}


// Unsigned division by an invariant d for dividends below 2^31 (the round-up multiply
// and shift of Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994): q = (mulhi(n, m) + n) >> l with l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1. The host checks it over the dividends a plan uses.
struct FastDiv {
    uint32_t d, m, l;
};

__host__ __device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv &f) {
#ifdef __CUDA_ARCH__
    return (__umulhi(n, f.m) + n) >> f.l;
#else
    return (uint32_t)((((uint64_t)n * f.m) >> 32) + n) >> f.l;
#endif
}

struct MixedArgs {
    PassParams p;            // buffers, planes, line / element strides, conj, stage table (tw),
                             // inter-pass diagonal (tw2_full, columns kind), error word
    int32_t L, C, nst, pitch;
    int32_t lpt;             // lines per transform (1 rows, K columns, M transposed rows)
    int32_t flat;            // FP32 split single pass: move the tile with flat vector copies
    FastDiv div_lpt, div_L, div_C;
    int8_t radix[kMixedMaxStages];
    int32_t ns[kMixedMaxStages], tw_off[kMixedMaxStages];
    FastDiv div_lr[kMixedMaxStages], div_ns[kMixedMaxStages];
};

// cos and sin of 2 pi m / r for the odd radices (mathematical constants)
__host__ __device__ constexpr float mixed_cos(int r, int m) {
    return r == 3 ? (m == 1 ? -0.5f : -0.5f)
         : r == 5 ? (m == 1 ? 0.30901699437494742410f : -0.80901699437494742410f)
                  : (m == 1 ? 0.62348980185873353053f : m == 2 ? -0.22252093395631440429f : -0.90096886790241912624f);
}
__host__ __device__ constexpr float mixed_sin(int r, int m) {
    return r == 3 ? 0.86602540378443864676f
         : r == 5 ? (m == 1 ? 0.95105651629515357212f : 0.58778525229247312917f)
                  : (m == 1 ? 0.78183148246802980871f : m == 2 ? 0.97492791218182360702f : 0.43388373911755812048f);
}

// Forward DFT_R for odd prime R in registers: with a_j = x_j + x_{R-j} and
// b_j = x_j - x_{R-j} (j = 1 .. (R-1)/2),
//   X_k     = x_0 + sum_j cos(2 pi jk/R) a_j - i sum_j sin(2 pi jk/R) b_j
//   X_{R-k} = x_0 + sum_j cos(2 pi jk/R) a_j + i sum_j sin(2 pi jk/R) b_j.
// odd-radix constants: FP32 from the pinned literals, FP64 from the compile-time series
template <typename V>
__host__ __device__ constexpr typename CplxT<V>::S odd_cos(int r, int m) {
    return std::is_same<V, float2>::value ? (typename CplxT<V>::S)mixed_cos(r, m) : (typename CplxT<V>::S)ct_cos(m, r);
}
template <typename V>
__host__ __device__ constexpr typename CplxT<V>::S odd_sin(int r, int m) {
    return std::is_same<V, float2>::value ? (typename CplxT<V>::S)mixed_sin(r, m) : (typename CplxT<V>::S)ct_sin(m, r);
}

template <int R, typename V>
__device__ __forceinline__ void dft_odd(V *x) {
    using S = typename CplxT<V>::S;
    constexpr int H = (R - 1) / 2;
    V a[H + 1], b[H + 1];
    V s0 = x[0];
#pragma unroll
    for (int j = 1; j <= H; ++j) {
        a[j] = cadd(x[j], x[R - j]);
        b[j] = csub(x[j], x[R - j]);
        s0 = cadd(s0, a[j]);
    }
    V y[R];
    y[0] = s0;
#pragma unroll
    for (int k = 1; k <= H; ++k) {
        V A = x[0], B = CplxT<V>::make(0, 0);
#pragma unroll
        for (int j = 1; j <= H; ++j) {
            const int m = (j * k) % R;  // compile-time
            const S c = m <= H ? odd_cos<V>(R, m) : odd_cos<V>(R, R - m);
            const S s = m <= H ? odd_sin<V>(R, m) : -odd_sin<V>(R, R - m);
            A.x += c * a[j].x;
            A.y += c * a[j].y;
            B.x += s * b[j].x;
            B.y += s * b[j].y;
        }
        // -i B = (B.y, -B.x)
        y[k] = CplxT<V>::make(A.x + B.y, A.y - B.x);
        y[R - k] = CplxT<V>::make(A.x - B.y, A.y + B.x);
    }
#pragma unroll
    for (int k = 0; k < R; ++k) x[k] = y[k];
}

__host__ __device__ constexpr int ct_spf(int r) { return r % 2 == 0 ? 2 : r % 3 == 0 ? 3 : r % 5 == 0 ? 5 : r % 7 == 0 ? 7 : r; }

// x *= w_R^e (forward, w_R = exp(-2 pi i / R)) with a compile-time exponent: quarter turns
// exactly, other angles from the compile-time cos / sin
template <int R, int E, typename V>
__device__ __forceinline__ V mul_wr(V x) {
    using S = typename CplxT<V>::S;
    constexpr int e = E % R;
    if constexpr (e == 0) {
        return x;
    } else if constexpr ((4 * e) % R == 0) {
        constexpr int q = 4 * e / R;  // quarter turns
        if constexpr (q == 1) return CplxT<V>::make(x.y, -x.x);
        else if constexpr (q == 2) return CplxT<V>::make(-x.x, -x.y);
        else return CplxT<V>::make(-x.y, x.x);
    } else {
        constexpr S c = (S)ct_cos(e, R), s = (S)ct_sin(e, R);
        return CplxT<V>::make(x.x * c + x.y * s, x.y * c - x.x * s);
    }
}

template <int R, typename V>
__device__ __forceinline__ void dft_small(V *v);

// DFT_R for composite R = P Q in registers (Eq. 1 once more): input j = a + P b; the Q-point
// DFTs over b for every a, the twiddles w_R^(a q), then the P-point DFTs over a, giving
// output q + Q k
template <int P, int Q, int A, typename V, int q = 0>
__device__ __forceinline__ void ct_scatter(V *v, const V *t) {
    if constexpr (q < Q) {
        v[A + P * q] = mul_wr<P * Q, A * q>(t[q]);
        ct_scatter<P, Q, A, V, q + 1>(v, t);
    }
}

template <int P, int Q, typename V, int A = 0>
__device__ __forceinline__ void ct_inner(V *v) {
    if constexpr (A < P) {
        V t[Q];
#pragma unroll
        for (int b = 0; b < Q; ++b) t[b] = v[A + P * b];
        dft_small<Q>(t);
        ct_scatter<P, Q, A, V>(v, t);
        ct_inner<P, Q, V, A + 1>(v);
    }
}

template <int P, int Q, typename V>
__device__ __forceinline__ void dft_ct(V *v) {
    ct_inner<P, Q, V>(v);
    V y[P * Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        V u[P];
#pragma unroll
        for (int a = 0; a < P; ++a) u[a] = v[a + P * q];
        dft_small<P>(u);
#pragma unroll
        for (int k = 0; k < P; ++k) y[q + Q * k] = u[k];
    }
#pragma unroll
    for (int i = 0; i < P * Q; ++i) v[i] = y[i];
}

template <int R, typename V>
__device__ __forceinline__ void dft_small(V *v) {
    if constexpr (R == 1) {
        return;
    } else if constexpr (R == 2) {
        const V a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr ((R & (R - 1)) == 0 && std::is_same<V, float2>::value) {
        dft<R>(v);  // FP32: the radix-2 network with its exact constant twiddles
    } else if constexpr (ct_spf(R) == R) {
        dft_odd<R>(v);
    } else {
        dft_ct<ct_spf(R), R / ct_spf(R), V>(v);
    }
}

// One stage over the tile. IO bit 0: the stage reads HBM (the first stage), bit 1: it writes
// HBM (the last stage); otherwise shared memory. Line g0 + c, element e sits at
// (g / lpt) tr + (g mod lpt) line + e elem. CF: consecutive threads take consecutive lines
// at one position (coalesced for column access: the four-step pass 1 reads and writes, and
// pass 2's transposed writes); else consecutive positions of one line. KIND_COLS multiplies
// its output by the inter-pass diagonal (when the plan has one).
// CT_L > 0: the line length, lines per tile (CT_C), line pitch in shared memory (CT_P) and
// this stage's Ns (CT_NS) are compile-time constants (the per-length kernels of
// k_mixed_ct): every division, index product and loop bound of the stage is then resolved
// by the compiler.
template <int R, int NT, typename V, int IO = 0, int LIN = LAYOUT_IL, int LOUT = LAYOUT_IL, int KIND = KIND_ROWS,
          bool CF = false, int CT_L = 0, int CT_C = 0, int CT_NS = 0, int CT_P = 0>
__device__ __forceinline__ void mixed_stage(const MixedArgs &a, int s, const V *src, V *dst, int64_t g0 = 0) {
    using S = typename CplxT<V>::S;
    const PassParams &p = a.p;
    const int L = CT_L ? CT_L : a.L, Lr = L / R, Ns = CT_L ? CT_NS : a.ns[s];
    const int C = CT_L ? CT_C : a.C, pitch = CT_L ? CT_P : a.pitch;
    const int G = C * Lr;
    const V *tw = reinterpret_cast<const V *>(p.tw) + a.tw_off[s];
#pragma unroll 2
    for (int gi = threadIdx.x; gi < G; gi += NT) {
        int c, j;
        if constexpr (CT_L > 0) {
            if constexpr (CF) {
                j = gi / C;
                c = gi - j * C;
            } else {
                c = gi / Lr;
                j = gi - c * Lr;
            }
        } else if constexpr (CF) {
            j = (int)fdiv((uint32_t)gi, a.div_C);
            c = gi - j * a.C;
        } else {
            c = (int)fdiv((uint32_t)gi, a.div_lr[s]);
            j = gi - c * Lr;
        }
        V v[R];
        int64_t tr = 0, l = 0;
        bool live = true;
        if constexpr ((IO & 3) != 0) {
            const int64_t g = g0 + c;
            live = g < p.total_lines;
            tr = fdiv((uint32_t)g, a.div_lpt);
            l = g - tr * a.lpt;
        }
        if constexpr (IO & 1) {
            const int64_t b = tr * p.in_tr + l * p.in_line + (int64_t)j * p.in_elem;
            const S *pin = reinterpret_cast<const S *>(p.in);
#pragma unroll
            for (int t = 0; t < R; ++t) {
                V x = CplxT<V>::make(0, 0);
                if (live) {
                    const int64_t o = b + (int64_t)t * Lr * p.in_elem;
                    if constexpr (LIN == LAYOUT_IL) {
                        x = __ldcs(reinterpret_cast<const V *>(pin) + o);
                    } else {
                        x.x = __ldcs(pin + o);
                        x.y = __ldcs(pin + p.in_plane + o);
                    }
                }
                if (p.conj_in) x.y = -x.y;
                v[t] = x;
            }
        } else {
            const V *line = src + c * pitch;
#pragma unroll
            for (int t = 0; t < R; ++t) v[t] = line[j + t * Lr];
        }
        const int jq = CT_L ? j / Ns : (int)fdiv((uint32_t)j, a.div_ns[s]);
        const int jm = j - jq * Ns;
        if (Ns > 1) {
#pragma unroll
            for (int t = 1; t < R; ++t) v[t] = cmul(v[t], __ldg(tw + (t - 1) * Ns + jm));
        }
        dft_small<R>(v);
        const int o = jq * Ns * R + jm;
        if constexpr (IO & 2) {
            if (live) {
                const int64_t b = tr * p.out_tr + l * p.out_line;
                S *pout = reinterpret_cast<S *>(p.out);
#pragma unroll
                for (int t = 0; t < R; ++t) {
                    V x = v[t];
                    const int e = o + t * Ns;
                    if constexpr (KIND == KIND_COLS) {  // inter-pass diagonal: column l, row e
                        if (p.tw2_full) x = cmul(x, __ldg(reinterpret_cast<const V *>(p.tw2_full) + (int64_t)e * a.lpt + l));
                    }
                    if (p.post_h) {  // the fused diagonal: frequency l * line_mul + e * elem_mul
                        const S h = (S)(__ldg(p.post_h + l * p.post_line_mul + (int64_t)e * p.post_elem_mul) *
                                        p.post_scale);
                        x.x *= h;
                        x.y *= h;
                    }
                    if (p.conj_out) x.y = -x.y;
                    const int64_t q = b + (int64_t)e * p.out_elem;
                    if constexpr (KIND == KIND_COLS && LOUT == LAYOUT_IL) {
                        __stcg(reinterpret_cast<V *>(pout) + q, x);  // workspace: keep it in L2
                    } else if constexpr (LOUT == LAYOUT_IL) {
                        __stcs(reinterpret_cast<V *>(pout) + q, x);
                    } else {
                        __stcs(pout + q, x.x);
                        __stcs(pout + p.out_plane + q, x.y);
                    }
                }
            }
        } else {
            V *out = dst + c * pitch;
#pragma unroll
            for (int t = 0; t < R; ++t) out[o + t * Ns] = v[t];
        }
    }
}

template <int NT, typename V, int IO = 0, int LIN = LAYOUT_IL, int LOUT = LAYOUT_IL, int KIND = KIND_ROWS,
          bool CF = false>
__device__ __forceinline__ void run_stage(const MixedArgs &a, int s, const V *src, V *dst, int64_t g0 = 0) {
    switch (a.radix[s]) {
        case 2: mixed_stage<2, NT, V, IO, LIN, LOUT, KIND, CF>(a, s, src, dst, g0); break;
        case 3: mixed_stage<3, NT, V, IO, LIN, LOUT, KIND, CF>(a, s, src, dst, g0); break;
        case 4: mixed_stage<4, NT, V, IO, LIN, LOUT, KIND, CF>(a, s, src, dst, g0); break;
        case 5: mixed_stage<5, NT, V, IO, LIN, LOUT, KIND, CF>(a, s, src, dst, g0); break;
        case 6: mixed_stage<6, NT, V, IO, LIN, LOUT, KIND, CF>(a, s, src, dst, g0); break;
        case 7: mixed_stage<7, NT, V, IO, LIN, LOUT, KIND, CF>(a, s, src, dst, g0); break;
        case 8: mixed_stage<8, NT, V, IO, LIN, LOUT, KIND, CF>(a, s, src, dst, g0); break;
        case 9: mixed_stage<9, NT, V, IO, LIN, LOUT, KIND, CF>(a, s, src, dst, g0); break;
        case 10: mixed_stage<10, NT, V, IO, LIN, LOUT, KIND, CF>(a, s, src, dst, g0); break;
        case 12: mixed_stage<12, NT, V, IO, LIN, LOUT, KIND, CF>(a, s, src, dst, g0); break;
        case 14: mixed_stage<14, NT, V, IO, LIN, LOUT, KIND, CF>(a, s, src, dst, g0); break;
        case 15: mixed_stage<15, NT, V, IO, LIN, LOUT, KIND, CF>(a, s, src, dst, g0); break;
        default: mixed_stage<16, NT, V, IO, LIN, LOUT, KIND, CF>(a, s, src, dst, g0); break;
    }
}

// Single pass, FP32 split layout: the tile's lines are back to back in both planes, so the
// first stage's input and the last stage's output move as flat 16-byte vectors per plane
// through shared memory (pitch L) when the tile starts 16-byte aligned in both planes.
template <int LAY, int NT, bool LOAD>
__device__ __forceinline__ void rows_copy(const MixedArgs &a, int64_t g0, float2 *sm) {
    const PassParams &p = a.p;
    const int64_t lines = min((int64_t)a.C, p.total_lines - g0);
    const int T = (int)lines * a.L;
    const int64_t base = g0 * a.L;  // element offset of the tile (in_tr = out_tr = L)
    const int cj = LOAD ? p.conj_in : p.conj_out;
    constexpr int V = LAY == LAYOUT_IL ? 2 : 4;  // elements per 16-byte vector and plane
    int done = 0;
    const int64_t plane = LAY == LAYOUT_IL ? 0 : (LOAD ? p.in_plane : p.out_plane);
    if (((base | plane) & (V - 1)) == 0) {
        const int nv = T / V;
        if constexpr (LAY == LAYOUT_IL) {
            float4 *g = reinterpret_cast<float4 *>((LOAD ? const_cast<float *>(p.in) : p.out) + 2 * base);
            float4 *sv = reinterpret_cast<float4 *>(sm);
#pragma unroll 8
            for (int u = threadIdx.x; u < nv; u += NT) {
                if constexpr (LOAD) {
                    float4 q = __ldcs(g + u);
                    if (cj) {
                        q.y = -q.y;
                        q.w = -q.w;
                    }
                    sv[u] = q;
                } else {
                    float4 q = sv[u];
                    if (cj) {
                        q.y = -q.y;
                        q.w = -q.w;
                    }
                    __stcs(g + u, q);
                }
            }
        } else {
            float *pl = LOAD ? const_cast<float *>(p.in) : p.out;
            float4 *gr = reinterpret_cast<float4 *>(pl + base), *gi = reinterpret_cast<float4 *>(pl + plane + base);
#pragma unroll 4
            for (int u = threadIdx.x; u < nv; u += NT) {
                float2 *e = sm + 4 * u;
                if constexpr (LOAD) {
                    const float4 r = __ldcs(gr + u), i = __ldcs(gi + u);
                    const float sg = cj ? -1.f : 1.f;
                    e[0] = make_float2(r.x, sg * i.x);
                    e[1] = make_float2(r.y, sg * i.y);
                    e[2] = make_float2(r.z, sg * i.z);
                    e[3] = make_float2(r.w, sg * i.w);
                } else {
                    const float sg = cj ? -1.f : 1.f;
                    __stcs(gr + u, make_float4(e[0].x, e[1].x, e[2].x, e[3].x));
                    __stcs(gi + u, make_float4(sg * e[0].y, sg * e[1].y, sg * e[2].y, sg * e[3].y));
                }
            }
        }
        done = nv * V;
    }
    for (int f = done + (int)threadIdx.x; f < T; f += NT) {  // unaligned tile or vector tail
        if constexpr (LOAD) {
            float2 x;
            if constexpr (LAY == LAYOUT_IL) {
                x = __ldcs(reinterpret_cast<const float2 *>(p.in) + base + f);
            } else {
                x.x = __ldcs(p.in + base + f);
                x.y = __ldcs(p.in + p.in_plane + base + f);
            }
            if (cj) x.y = -x.y;
            sm[f] = x;
        } else {
            float2 x = sm[f];
            if (cj) x.y = -x.y;
            if constexpr (LAY == LAYOUT_IL) {
                __stcs(reinterpret_cast<float2 *>(p.out) + base + f, x);
            } else {
                __stcs(p.out + base + f, x.x);
                __stcs(p.out + p.out_plane + base + f, x.y);
            }
        }
    }
}

template <int KIND, int LIN, int LOUT, int NT, typename V>
__global__ void __launch_bounds__(NT) k_mixed(const __grid_constant__ MixedArgs a) {
    extern __shared__ __align__(16) unsigned char sm_mixed_raw[];
    V *sm_mixed = reinterpret_cast<V *>(sm_mixed_raw);
    V *buf0 = sm_mixed, *buf1 = sm_mixed + ((a.C * a.pitch + 1) & ~1);
    const int64_t g0 = (int64_t)blockIdx.x * a.C;
    if constexpr (KIND == KIND_ROWS) {
        // single pass: the first stage reads HBM and the last writes it (lines back to back)
        // (FP32 split with short lines: through shared memory with 16-byte vectors per plane,
        // where the scalar 4-byte plane accesses of the direct stages cost more)
        bool flat = false;
        // (not with the fused diagonal, which the direct last stage applies)
        if constexpr (std::is_same<V, float2>::value && LIN == LAYOUT_SPLIT) flat = a.flat != 0 && !a.p.post_h;
        if (flat) {
            if constexpr (std::is_same<V, float2>::value && LIN == LAYOUT_SPLIT) rows_copy<LIN, NT, true>(a, g0, buf1);
            __syncthreads();
        } else if (a.nst == 1) {
            run_stage<NT, V, 3, LIN, LOUT>(a, 0, nullptr, nullptr, g0);
            return;
        }
        V *src = buf0, *dst = buf1;
        if (flat) run_stage<NT, V>(a, 0, buf1, buf0);
        else run_stage<NT, V, 1, LIN, LOUT>(a, 0, nullptr, buf0, g0);
        __syncthreads();
        const int last = flat ? a.nst : a.nst - 1;
        for (int s = 1; s < last; ++s) {
            run_stage<NT, V>(a, s, src, dst);
            __syncthreads();
            V *t = src;
            src = dst;
            dst = t;
        }
        if (flat) {
            if constexpr (std::is_same<V, float2>::value && LIN == LAYOUT_SPLIT) rows_copy<LOUT, NT, false>(a, g0, src);
        } else {
            run_stage<NT, V, 2, LIN, LOUT>(a, a.nst - 1, src, nullptr, g0);
        }
    } else {
        // four-step passes and strided axes: pass 1 (columns) reads and writes line-fastest;
        // pass 2 reads its contiguous rows position-fastest and writes transposed line-fastest
        constexpr bool CF_IN = KIND == KIND_COLS, CF_OUT = true;
        if (a.nst == 1) {
            run_stage<NT, V, 3, LIN, LOUT, KIND, CF_IN>(a, 0, nullptr, nullptr, g0);
            return;
        }
        run_stage<NT, V, 1, LIN, LOUT, KIND, CF_IN>(a, 0, nullptr, buf0, g0);
        __syncthreads();
        V *src = buf0, *dst = buf1;
        for (int s = 1; s < a.nst - 1; ++s) {
            run_stage<NT, V>(a, s, src, dst);
            __syncthreads();
            V *t = src;
            src = dst;
            dst = t;
        }
        run_stage<NT, V, 2, LIN, LOUT, KIND, CF_OUT>(a, a.nst - 1, src, nullptr, g0);
    }
}

}  // namespace fftc

namespace fftc {

// kernel variants of one element type: [kind and layouts][CTA of 512 threads]
typedef void (*MixedKernel)(MixedArgs);
enum { MK_ROWS_IL, MK_ROWS_SPLIT, MK_COLS_IL, MK_COLS_SPLIT_IL, MK_COLS_SPLIT, MK_ROWST_IL, MK_ROWST_SPLIT, MK_COUNT };
struct MixedKernelSet {
    MixedKernel k[MK_COUNT][2];
};

}  // namespace fftc

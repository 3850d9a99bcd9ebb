// The fused Stockham pass kernel.
//
// One CTA transforms C lines of length L = 2^LOGL held in registers (E = 2^LOGE
// complex values per thread) and exchanged through shared memory between radix
// stages. Each stage is one factor of the paper's Eq. 1 applied to every
// sub-transform at once:
//   read   a[t] = x[j + t L/R]                      (the stride permutation Pi)
//   twiddle a[t] *= w_{Ns R}^{t (j mod Ns)}          (the diagonal D, Table 1 "Mul")
//   butterfly a = DFT_R a                            (I (x) DFT_R, Table 1 FusedIKMV/MKIV)
//   write  y[(j/Ns) Ns R + j mod Ns + t Ns] = a[t]   (Stockham autosort)
// The first stage reads HBM directly and the last one writes HBM directly, both
// coalesced, so one pass moves each element through HBM once.
//
// Shared-memory layout. Stage 0 has radix E and Ns = 1, so its writes land on
// j E + t, E words apart across threads: the first exchange therefore stores word a
// at a + (a >> LOGE) (one skew word per E words). Every later stage has Ns >= E >= 16
// and writes runs of consecutive words, so later exchanges use the identity layout.
// With both layouts every shared access of a thread is a per-thread base plus a
// compile-time offset, and a half-warp touches 16 distinct banks (checked with a bank
// simulator for E = 16, L >= 256 and E = 32, L >= 512).
//
// Thread <-> (line c, position tau) mapping, chosen per stage:
//   tau-fast: consecutive threads walk one line (coalesced for contiguous lines);
//   c-fast:   consecutive threads walk C lines at the same position (coalesced for
//             column access at unit line stride; the line pitch keeps it conflict-free).
//
// Element strides: 1 for contiguous lines; for the four-step passes the stride is
// the other factor 2^LOGX of n = M K, a compile-time constant when LOGX > 0.
#pragma once

#include <algorithm>

#include "fftc_device.cuh"
#include "fftc_internal.h"
#include "fftc_tc.cuh"

namespace fftc {

// Line pitch in float2 words: odd for 16-line tiles (their c-fast accesses then hit 16
// distinct banks), +2 otherwise so that every line slot starts 16-byte aligned (a bulk
// copy destination) while the 8-line c-fast accesses stay conflict-free.
__host__ __device__ constexpr int pass_pitch(int line_words, int lines) {
    return lines == 1 ? line_words : line_words + (lines >= 16 ? 1 : 2);
}

// no-op tile hook (see Pass::run_tile_landed)
struct NoHook {
    static constexpr bool active = false;
    __device__ __forceinline__ void operator()() const {}
};

// 128-byte aligned start of dynamic shared memory (the tensor-core area when TC is set)
__device__ __forceinline__ unsigned char *dyn_smem_base128() {
    extern __shared__ __align__(16) unsigned char dyn_raw[];
    return dyn_raw + ((128 - (smem_u32(dyn_raw) & 127)) & 127);
}

template <int LOGL, int LOGE, int C, int KIND, int LIN, int LOUT, bool IDX = false, int LOGX = 0, int TCM = 0>
struct Pass {
    // TCM: 0 = every stage on the CUDA cores; 1..4 = the radix-E stages (E = 16 or 32) on the
    // tensor cores in that precision mode (TcMode)
    static constexpr bool TC = TCM != 0;
    static constexpr int TCM_ID = TCM;
    using Sc = Sched<LOGL, LOGE>;
    static constexpr int L = Sc::L, E = Sc::E, TPL = Sc::TPL, S = Sc::S;
    static constexpr int NT = C * TPL;
    static constexpr int C_LINES = C, LIN_LAYOUT = LIN, KIND_ID = KIND;
    static constexpr int LINE_WORDS = L + (L >> LOGE);
    static constexpr int PITCH = pass_pitch(LINE_WORDS, C);
    // TC: the radix-E stages (E = 16 or 32) on the tensor cores (fftc_tc.cuh); the
    // tensor-core area (DFT matrices, mbarriers) sits in front of the data in dynamic shared
    // memory; a shorter last stage runs on the CUDA cores
    static constexpr int TC_BYTES = TC ? tc_area_bytes(E) : 0;
    static constexpr int DATA_BYTES = (S > 1) ? C * PITCH * (int)sizeof(float2) : 0;
    static constexpr int SMEM = TC ? TC_BYTES + DATA_BYTES + 128 : DATA_BYTES;
    static_assert(!TC || ((LOGE == 4 || LOGE == 5) && NT % 128 == 0 && !IDX),
                  "tensor-core passes: 16 or 32 elements per thread");
    __host__ __device__ static constexpr int tc_count(int upto) {
        int c = 0;
        for (int i = 0; i < upto; ++i) c += (Sc::lr(i) == LOGE) ? 1 : 0;
        return c;
    }
    static constexpr int NTC = TC ? tc_count(S) : 0;  // tensor-core stages per tile
    __host__ __device__ static constexpr float tc_out_scale() {
        float f = 1.f;
        for (int i = 0; i < NTC; ++i) f *= 4.f;
        return f;
    }
    static constexpr bool COLS_LIKE = (KIND == KIND_COLS || KIND == KIND_CLUSTER_A);
    static constexpr bool IN_TAU = !COLS_LIKE;
    static constexpr bool OUT_TAU = (KIND == KIND_ROWS);
    static constexpr bool MID_TAU = (C < 16);
    static_assert(S > 1 || IN_TAU == OUT_TAU, "a single-stage pass cannot change its mapping");
    static_assert(NT >= 32 && NT <= 1024, "CTA size out of range");
    __host__ __device__ static constexpr bool tau_fast(int s) {
        return s == 0 ? IN_TAU : (s == S - 1 ? OUT_TAU : MID_TAU);
    }
    static constexpr bool all_tau() {
        for (int s = 0; s < S; ++s)
            if (!tau_fast(s)) return false;
        return true;
    }
    // a line never leaves one warp: warp-level barriers are enough
    static constexpr bool WARP_SYNC = all_tau() && TPL <= 32 && (32 % TPL) == 0;
    // registers per thread the launch bounds aim at: E = 32 needs ~128; E = 16 fits 80, or 64
    // for 512-thread CTAs so that two of them share an SM
    static constexpr int REG_TARGET = TC ? (E >= 32 ? 128 : 64) : (E >= 32 ? 128 : (E >= 16 ? (NT >= 512 ? 64 : 80) : 64));
    static constexpr int MINB = (65536 / (NT * REG_TARGET)) > 0 ? (65536 / (NT * REG_TARGET)) : 1;
    // element strides: compile-time unless LOGX == 0 for a four-step kind
    static constexpr int ES_IN_CT = COLS_LIKE ? (LOGX ? (1 << LOGX) : 0) : 1;
    static constexpr int ES_OUT_CT = (KIND == KIND_ROWS) ? 1 : (LOGX ? (1 << LOGX) : 0);
    // the four-step workspace is written in the same launch in persistent mode: read it
    // from L2 only, never through a possibly stale L1 line
    static constexpr bool IN_L2ONLY = (KIND == KIND_ROWST);

    __device__ __forceinline__ static void sync() {
        if constexpr (WARP_SYNC)
            __syncwarp();
        else
            __syncthreads();
    }

    __device__ __forceinline__ static int64_t line_off(const PassParams &p, int64_t g, int64_t tr, int64_t line) {
        if constexpr (IDX) return __ldg(p.line_off + g);
        return (g >> p.log_lpt) * tr + (g & ((int64_t(1) << p.log_lpt) - 1)) * line;
    }
    __device__ __forceinline__ static int conj_of(const PassParams &p, int64_t g, int flag) {
        if constexpr (IDX) return __ldg(p.line_conj + g);
        return flag;
    }

    template <int R>
    __device__ __forceinline__ static void load_global(const PassParams &p, float2 (&v)[E], int tau, int64_t g,
                                                       bool live) {
        const int64_t base = line_off(p, g, p.in_tr, p.in_line);
        const int cj = conj_of(p, g, p.conj_in);
        const int es = ES_IN_CT ? ES_IN_CT : (int)p.in_elem;
#pragma unroll
        for (int q = 0; q < E / R; ++q) {
            const int64_t b = base + (int64_t)(tau + q * TPL) * es;
            const float2 *p2 = reinterpret_cast<const float2 *>(p.in) + b;
            const float *pr = p.in + b, *pi = p.in + p.in_plane + b;
#pragma unroll
            for (int t = 0; t < R; ++t) {
                const int off = t * (L / R) * es;  // compile-time when the stride is
                float2 x = make_float2(0.f, 0.f);
                if (live) {
                    if constexpr (LIN == LAYOUT_IL) {
                        if constexpr (IN_L2ONLY) x = __ldcg(p2 + off);
                        else x = __ldcs(p2 + off);
                    } else {
                        x.x = __ldcs(pr + off);
                        x.y = __ldcs(pi + off);
                    }
                }
                if (cj) x.y = -x.y;
                v[q * R + t] = x;
            }
        }
    }

    template <int R>
    __device__ __forceinline__ static void store_global(const PassParams &p, float2 (&v)[E], int tau, int64_t g,
                                                        bool live) {
        if (!live) return;
        const int l = (int)(g & ((int64_t(1) << p.log_lpt) - 1));
        const int64_t base = line_off(p, g, p.out_tr, p.out_line);
        const int cj = conj_of(p, g, p.conj_out);
        const int es = ES_OUT_CT ? ES_OUT_CT : (int)p.out_elem;
        const float2 *dtab = nullptr;
        if constexpr (COLS_LIKE) dtab = p.tw2_full ? p.tw2_full + l * (int)p.out_line : nullptr;
#pragma unroll
        for (int q = 0; q < E / R; ++q) {
            const int a0 = tau + q * TPL;
            const int64_t b = base + (int64_t)a0 * es;
            float2 *p2 = reinterpret_cast<float2 *>(p.out) + b;
            float *pr = p.out + b, *pi = p.out + p.out_plane + b;
#pragma unroll
            for (int t = 0; t < R; ++t) {
                const int off = t * (L / R) * es;
                float2 x = v[q * R + t];
                if constexpr (COLS_LIKE) {
                    // inter-pass twiddle of Eq. 1 applied at the memory level: w_N^(b t')
                    if (dtab) {
                        x = cmul(x, __ldg(dtab + a0 * es + off));
                    } else if (p.tw2_lo) {  // none for a strided axis of a multidimensional array
                        const int a = a0 + t * (L / R);
                        const int m = (l * a) & ((1 << p.log_n2) - 1);
                        x = cmul(x, cmul(__ldg(p.tw2_lo + (m & ((1 << p.tw2_lo_bits) - 1))),
                                         __ldg(p.tw2_hi + (m >> p.tw2_lo_bits))));
                    }
                }
                if constexpr (TC && !tc_is_bf16(TCM)) {
                    {  // FP16 stages ran on data scaled by 1/4 each
                        x.x *= tc_out_scale();
                        x.y *= tc_out_scale();
                    }
                }
                if (p.post_h) {
                    const int a = a0 + t * (L / R);
                    const float h = __ldg(p.post_h + l * (int)p.post_line_mul + a * (int)p.post_elem_mul) * p.post_scale;
                    x.x *= h;
                    x.y *= h;
                }
                if (cj) x.y = -x.y;
                if constexpr (KIND == KIND_CLUSTER_A) {
                    // output a of column l goes to row a mod Qb of the CTA that owns rows
                    // [a - a mod Qb, + Qb) in phase B, position l of that row (row-major)
                    const int a = a0 + t * (L / R);
                    const uint32_t rank = (uint32_t)(a >> p.cl_log_rows);
                    const uint32_t word = (uint32_t)(((a & ((1 << p.cl_log_rows) - 1)) << p.log_lpt) + l);
                    st_cluster_v2(mapa_shared(smem_u32(dyn_smem_base128()) + 8u * word, rank), x.x, x.y);
                } else if constexpr (KIND == KIND_COLS && LOUT == LAYOUT_IL) {
                    __stcg(p2 + off, x);  // workspace: keep it in L2 for pass 2
                } else if constexpr (LOUT == LAYOUT_IL) {
                    __stcs(p2 + off, x);
                } else {
                    __stcs(pr + off, x.x);
                    __stcs(pi + off, x.y);
                }
            }
        }
    }

    // Stage-0 operands from a landing buffer filled by the bulk-copy (TMA) engine:
    //   single pass (contiguous lines, one copy per line): line c in its PITCH slot,
    //     interleaved, or split as L reals then L imaginaries;
    //   pass 2 (C consecutive workspace rows, one copy per tile): row-major [c][a];
    //   pass 1 (a 2D tensor box of C columns x L rows): column-major [a][c], split as
    //     the real box then the imaginary box.
    __device__ __forceinline__ static float2 landed(const float2 *sm, int c, int a) {
        if constexpr (KIND == KIND_ROWS) {
            if constexpr (LIN == LAYOUT_IL) return sm[c * PITCH + a];
            const float *lf = reinterpret_cast<const float *>(sm + c * PITCH);
            return make_float2(lf[a], lf[L + a]);
        } else if constexpr (KIND == KIND_ROWST) {
            return sm[c * L + a];
        } else {
            if constexpr (LIN == LAYOUT_IL) return sm[a * C + c];
            const float *lf = reinterpret_cast<const float *>(sm);
            return make_float2(lf[a * C + c], lf[L * C + a * C + c]);
        }
    }

    template <int R>
    __device__ __forceinline__ static void load_landed(const PassParams &p, float2 (&v)[E], const float2 *sm, int c,
                                                       int tau, int64_t g) {
        const int cj = conj_of(p, g, p.conj_in);
#pragma unroll
        for (int q = 0; q < E / R; ++q) {
            const int j = tau + q * TPL;
#pragma unroll
            for (int t = 0; t < R; ++t) {
                float2 x = landed(sm, c, j + t * (L / R));
                if (cj) x.y = -x.y;
                v[q * R + t] = x;
            }
        }
    }

    // `tk`: how many tiles this CTA transformed before this one (tensor-core mbarrier phases)
    template <int s, bool LANDED = false, class H = NoHook>
    __device__ __forceinline__ static void stage(const PassParams &p, float2 *sm, float2 (&v)[E], int tid, int64_t g0,
                                                 const H &hook = H(), uint32_t tk = 0) {
        constexpr int LR = Sc::lr(s), R = 1 << LR, LNS = Sc::lns(s), NS = 1 << LNS;
        constexpr bool TF = tau_fast(s);
        constexpr bool TCS = TC && LR == LOGE;  // this stage's butterfly runs on the tensor cores
        const int c = TF ? tid / TPL : tid % C;
        const int tau = TF ? tid % TPL : tid / C;
        const int64_t g = g0 + c;
        const bool live = g < p.total_lines;
        float2 *line = sm + c * PITCH;

        if constexpr (s == 0) {
            if constexpr (LANDED) load_landed<R>(p, v, sm, c, tau, g);
            else load_global<R>(p, v, tau, g, live);
        } else {
#pragma unroll
            for (int q = 0; q < E / R; ++q) {
                const int j = tau + q * TPL;
                if constexpr (s == 1) {  // skewed layout of the first exchange (L/R is a multiple of E)
                    const float2 *src = line + j + (j >> LOGE);
#pragma unroll
                    for (int t = 0; t < R; ++t) v[q * R + t] = src[t * (L / R) + ((t * (L / R)) >> LOGE)];
                } else {
                    const float2 *src = line + j;
#pragma unroll
                    for (int t = 0; t < R; ++t) v[q * R + t] = src[t * (L / R)];
                }
            }
            if constexpr (H::active && s == S - 1) {
                __syncthreads();  // the last shared read of the tile is done: the buffer is free
                hook();
            }
            const float2 *tw = p.tw + Sc::tw_off(s);
#pragma unroll
            for (int q = 0; q < E / R; ++q) {
                const float2 *twk = tw + ((tau + q * TPL) & (NS - 1));
#pragma unroll
                for (int t = 1; t < R; ++t) v[q * R + t] = cmul(v[q * R + t], __ldg(twk + (t - 1) * NS));
            }
        }
        if constexpr (TCS) {
            // the i-th tensor-core stage of this CTA's k-th tile uses mbarrier phase (k NTC + i) mod 2
            const uint32_t phase = (tk * NTC + tc_count(s)) & 1u;
            TcUnit<NT, TCM, E>::dft(p, v, dyn_smem_base128(), phase);
        } else {
#pragma unroll
            for (int q = 0; q < E / R; ++q) dft<R>(v + q * R);
        }

        if constexpr (s < S - 1) {
            if constexpr (s > 0 || LANDED) sync();  // every read of this stage precedes any overwrite
#pragma unroll
            for (int q = 0; q < E / R; ++q) {
                const int j = tau + q * TPL;
                if constexpr (s == 0) {  // Ns = 1, R = E: word j E + t, skewed to j (E + 1) + t
                    float2 *dst = line + j * (E + 1);
#pragma unroll
                    for (int t = 0; t < R; ++t) dst[t] = v[q * R + t];
                } else {
                    float2 *dst = line + ((j >> LNS) << (LNS + LR)) + (j & (NS - 1));
#pragma unroll
                    for (int t = 0; t < R; ++t) dst[t * NS] = v[q * R + t];
                }
            }
            sync();
            stage<s + 1, LANDED>(p, sm, v, tid, g0, hook, tk);
        } else {
            store_global<R>(p, v, tau, g, live);
        }
    }

    // ask L2 to fetch the input rows of `tile` (pass 1: L rows of C adjacent columns),
    // one prefetch per 32-byte sector
    __device__ __forceinline__ static void prefetch_tile(const PassParams &p, int64_t tile) {
        const int64_t g0 = tile * C;
        if (g0 >= p.total_lines) return;
        const int64_t base = line_off(p, g0, p.in_tr, p.in_line);
        const int64_t es = ES_IN_CT ? ES_IN_CT : p.in_elem;
        if constexpr (LIN == LAYOUT_IL) {
            constexpr int SPR = (C * 8 + 31) / 32;  // sectors per row
            const char *b = reinterpret_cast<const char *>(p.in + 2 * base);
            for (int i = threadIdx.x; i < L * SPR; i += NT)
                prefetch_l2(b + (i / SPR) * es * 8 + (i % SPR) * 32);
        } else {
            constexpr int SPR = (C * 4 + 31) / 32;
            for (int i = threadIdx.x; i < 2 * L * SPR; i += NT) {
                const int h = i / (L * SPR), j = i % (L * SPR);
                prefetch_l2(reinterpret_cast<const char *>(p.in + h * p.in_plane + base + (j / SPR) * es) +
                            (j % SPR) * 32);
            }
        }
    }

    __device__ __forceinline__ static void run(const PassParams &p) {
        extern __shared__ float2 sm_dyn[];
        if constexpr (KIND == KIND_COLS && !IDX && !TC)
            if (p.pf_tiles > 0) prefetch_tile(p, (int64_t)blockIdx.x + p.pf_tiles);
        float2 v[E];
        if constexpr (TC) {
            // persistent: the set-up (DFT matrices, mbarriers, TMEM columns) is paid once per CTA
            unsigned char *area = dyn_smem_base128();
            float2 *sm = reinterpret_cast<float2 *>(area + TC_BYTES);
            TcUnit<NT, TCM, E>::setup(p, area);
            const int64_t ntiles = (p.total_lines + C - 1) / C;
            uint32_t tk = 0;
            for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++tk) {
                if constexpr (KIND == KIND_COLS)
                    if (p.pf_tiles > 0) prefetch_tile(p, tile + gridDim.x);  // this CTA's next tile
                stage<0>(p, sm, v, threadIdx.x, tile * C, NoHook(), tk);
                __syncthreads();  // the tile's last shared reads precede the next tile's A rows
            }
            TcUnit<NT, TCM, E>::teardown(area);
        } else {
            stage<0>(p, sm_dyn, v, threadIdx.x, (int64_t)blockIdx.x * C);
        }
    }

    // one tile (C lines starting at line tile * C) with the caller's shared memory
    __device__ __forceinline__ static void run_tile(const PassParams &p, int64_t tile, float2 *sm) {
        float2 v[E];
        stage<0>(p, sm, v, threadIdx.x, tile * C);
    }

    // one tile whose input lines already sit in `sm` (see landed()); `hook` runs once,
    // by every thread, as soon as the tile's last shared-memory read is done
    template <class H = NoHook>
    __device__ __forceinline__ static void run_tile_landed(const PassParams &p, int64_t tile, float2 *sm,
                                                           const H &hook = H(), uint32_t tk = 0) {
        float2 v[E];
        stage<0, true>(p, sm, v, threadIdx.x, tile * C, hook, tk);
    }
};

template <int LOGL, int LOGE, int C, int KIND, int LIN, int LOUT, int LOGX, int TCM = 0>
__global__ void __launch_bounds__(Pass<LOGL, LOGE, C, KIND, LIN, LOUT, false, LOGX, TCM>::NT,
                                  Pass<LOGL, LOGE, C, KIND, LIN, LOUT, false, LOGX, TCM>::MINB)
    k_pass(const __grid_constant__ PassParams p) {
    Pass<LOGL, LOGE, C, KIND, LIN, LOUT, false, LOGX, TCM>::run(p);
}

// CTAs of a kernel that fit on one SM at once. For kernels that allocate tensor memory
// (tmem_cols > 0) the runtime's occupancy query answers one CTA per SM, while the SM holds
// as many as its registers, shared memory, threads and 512 TMEM columns allow; those
// limits are counted here instead.
inline int resident_per_sm(const void *func, int threads, int dyn_smem, int tmem_cols) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, threads, dyn_smem) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 0;
    }
    if (tmem_cols <= 0) return per_sm;
    cudaFuncAttributes fa;
    int dev = 0, smem_sm = 0, regs_sm = 0, thr_sm = 0, resv = 0;
    if (cudaFuncGetAttributes(&fa, func) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess) {
        cudaGetLastError();
        return per_sm > 0 ? per_sm : 1;
    }
    const int regs = (fa.numRegs + 7) / 8 * 8;  // registers are allocated 256 per warp
    int n = thr_sm / threads;
    if (regs > 0) n = std::min(n, regs_sm / (regs * threads));
    n = std::min(n, smem_sm / (dyn_smem + (int)fa.sharedSizeBytes + resv));
    n = std::min(n, 512 / tmem_cols);
    return std::max(n, std::max(per_sm, 1));
}

// CTAs of a k_pass instance resident on the current device at once (0 if unknown)
template <int LOGL, int LOGE, int C, int KIND, int LIN, int LOUT, int LOGX, int TCM = 0>
int resident_ctas() {
    static int r = -1;
    if (r < 0) {
        using P = Pass<LOGL, LOGE, C, KIND, LIN, LOUT, false, LOGX, TCM>;
        int sms = 0, dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return 0;
        const int per_sm = resident_per_sm((const void *)k_pass<LOGL, LOGE, C, KIND, LIN, LOUT, LOGX, TCM>, P::NT,
                                           P::SMEM, TCM ? (int)tc_tmem_cols(P::NT, P::E) : 0);
        r = per_sm * sms;
    }
    return r;
}

template <int LOGL, int LOGE, int C, int KIND, int LIN, int LOUT, int LOGX, int TCM = 0>
cudaError_t launch_pass(const PassParams &p, cudaStream_t st) {
    using P = Pass<LOGL, LOGE, C, KIND, LIN, LOUT, false, LOGX, TCM>;
    const int64_t blocks = (p.total_lines + C - 1) / C;
    if (blocks <= 0) return cudaSuccess;
    if constexpr (TCM != 0) {  // persistent: one wave of CTAs walks the tiles
        const int res = resident_ctas<LOGL, LOGE, C, KIND, LIN, LOUT, LOGX, TCM>();
        if (res <= 0) return cudaErrorInvalidConfiguration;
        const unsigned grid = (unsigned)(blocks < res ? blocks : res);
        k_pass<LOGL, LOGE, C, KIND, LIN, LOUT, LOGX, TCM><<<grid, P::NT, P::SMEM, st>>>(p);
        return cudaGetLastError();
    }
    if (blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
    if constexpr (KIND == KIND_COLS) {
        if (p.pf_tiles < 0) {
            PassParams q = p;
            q.pf_tiles = resident_ctas<LOGL, LOGE, C, KIND, LIN, LOUT, LOGX, TCM>();
            k_pass<LOGL, LOGE, C, KIND, LIN, LOUT, LOGX, TCM><<<(unsigned)blocks, P::NT, P::SMEM, st>>>(q);
            return cudaGetLastError();
        }
    }
    k_pass<LOGL, LOGE, C, KIND, LIN, LOUT, LOGX, TCM><<<(unsigned)blocks, P::NT, P::SMEM, st>>>(p);
    return cudaGetLastError();
}

template <int LOGL, int LOGE, int C, int KIND, int LIN, int LOUT, int LOGX, int TCM = 0>
cudaError_t prepare_pass() {
    using P = Pass<LOGL, LOGE, C, KIND, LIN, LOUT, false, LOGX, TCM>;
    if (P::SMEM <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(k_pass<LOGL, LOGE, C, KIND, LIN, LOUT, LOGX, TCM>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, P::SMEM);
}

template <int LOGL, int LOGE, int C, int KIND, int LIN, int LOUT, int LOGX = 0, int TCM = 0>
constexpr KernelEntry entry() {
    using P = Pass<LOGL, LOGE, C, KIND, LIN, LOUT, false, LOGX, TCM>;
    return KernelEntry{KIND,
                       LOGL,
                       LOGE,
                       C,
                       LIN,
                       LOUT,
                       P::NT,
                       P::SMEM,
                       &launch_pass<LOGL, LOGE, C, KIND, LIN, LOUT, LOGX, TCM>,
                       &prepare_pass<LOGL, LOGE, C, KIND, LIN, LOUT, LOGX, TCM>,
                       TCM,
                       LOGX,
                       0};
}

}  // namespace fftc

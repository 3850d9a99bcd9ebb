// Pipelined persistent pass kernels: the bulk-copy (TMA) engine streams whole tiles
// into shared memory while the CTA transforms the previous tile.
//
// Each CTA owns NBUF landing buffers, each with one mbarrier. Tile k of a CTA goes to
// buffer k mod NBUF; thread 0 arms the barrier with the expected byte count and issues
// the copies:
//   single pass:  one cp.async.bulk per line (two per line for the split layout);
//   four-step 2:  one cp.async.bulk for the tile's C consecutive workspace rows;
//   four-step 1:  cp.async.bulk.tensor.2d boxes of C columns x up to 256 rows through a
//                 tensor map of the input (one map per plane in the split layout).
// The CTA waits on the barrier (bounded: an expired wait sets the plan's error word,
// waits a bounded time for its own copies still in flight, and returns), transforms the
// tile with stage 0 reading the landed data and the exchanges reusing the same buffer,
// writes the result to HBM from registers, and only then refills the buffer with tile
// k + NBUF. So NBUF - 1 tiles of HBM reads are in flight behind the compute.
//
// EARLY variant: the refill is issued as soon as the tile's last shared-memory read is
// done, before its last radix stage and its HBM stores, so even NBUF = 1 keeps one tile's
// reads in flight behind the end of the previous tile; this lets a 135 KB tile (one CTA
// per SM) or two 68 KB tiles per SM overlap their loads with compute.
// (A per-thread 16-byte cp.async feed of the narrow pass-1 column bands measured slower
// than plain loads into registers, and tensor-map boxes of 64-byte rows slower still.)
#pragma once

#include <cuda.h>

#include "fftc_pass.cuh"
#include "fftc_ptx.cuh"

namespace fftc {

struct PipeArgs {
    PassParams p;
    CUtensorMap tm[2];  // four-step pass 1: input (real plane / interleaved) and imaginary plane
};

template <class P, int NBUF, bool EARLY = false>
struct PipeTile {
    static_assert(P::S > 1, "pipelined tiles need an exchange buffer");
    static constexpr int KIND = P::KIND_ID;
    static constexpr int C = P::C_LINES, L = P::L;
    static constexpr int RAW_WORDS = C * P::PITCH > C * L ? C * P::PITCH : C * L;
    static constexpr int BUF_WORDS = (RAW_WORDS + 15) / 16 * 16;  // 128-byte multiple
    // + room to align the base, + the tensor-core area in front of the buffers (TC passes)
    static constexpr int SMEM = NBUF * BUF_WORDS * (int)sizeof(float2) + 128 + P::TC_BYTES;
    static constexpr int NT = P::NT;
    static constexpr int BOXR = L < 256 ? L : 256;  // rows per tensor box (box dims <= 256)

    // thread 0: arm `bar` and start the copies of `tile` into `buf`
    __device__ __forceinline__ static void issue(const PipeArgs &a, int64_t tile, float2 *buf, uint64_t *bar) {
        const PassParams &p = a.p;
        if (p.test_no_copy) return;  // test hook: the barrier is never armed, its wait runs out
        const int64_t g0 = tile * C;
        if constexpr (P::COLS_LIKE) {
            const int tr = (int)(g0 >> p.log_lpt), b0 = (int)(g0 & ((int64_t(1) << p.log_lpt) - 1));
            mbar_arrive_expect_tx(bar, (uint32_t)(L * C * sizeof(float2)));
#pragma unroll
            for (int k = 0; k < L / BOXR; ++k) {
                const int y = tr * L + k * BOXR;
                if constexpr (P::LIN_LAYOUT == LAYOUT_IL) {
                    tensor2d_g2s(buf + k * BOXR * C, &a.tm[0], b0, y, bar);
                } else {
                    float *bf = reinterpret_cast<float *>(buf);
                    tensor2d_g2s(bf + k * BOXR * C, &a.tm[0], b0, y, bar);
                    tensor2d_g2s(bf + L * C + k * BOXR * C, &a.tm[1], b0, y, bar);
                }
            }
        } else if constexpr (KIND == KIND_ROWST) {
            // C consecutive rows of one transform are contiguous in the workspace
            const int64_t off = (g0 >> p.log_lpt) * p.in_tr + (g0 & ((int64_t(1) << p.log_lpt) - 1)) * p.in_line;
            constexpr uint32_t bytes = (uint32_t)(C * L * sizeof(float2));
            mbar_arrive_expect_tx(bar, bytes);
            bulk_g2s(buf, reinterpret_cast<const float2 *>(p.in) + off, bytes, bar);
        } else {
            const int64_t left = p.total_lines - g0;
            const int nl = left < C ? (int)left : C;
            constexpr uint32_t line_bytes = L * sizeof(float2);
            mbar_arrive_expect_tx(bar, line_bytes * nl);
            for (int c = 0; c < nl; ++c) {
                const int64_t off = (g0 + c) * p.in_tr;  // contiguous lines
                float2 *dst = buf + c * P::PITCH;
                if constexpr (P::LIN_LAYOUT == LAYOUT_IL) {
                    bulk_g2s(dst, reinterpret_cast<const float2 *>(p.in) + off, line_bytes, bar);
                } else {
                    float *df = reinterpret_cast<float *>(dst);
                    bulk_g2s(df, p.in + off, line_bytes / 2, bar);
                    bulk_g2s(df + L, p.in + p.in_plane + off, line_bytes / 2, bar);
                }
            }
        }
    }

    // refill `buf` with `tile`: called by every thread after a block-wide barrier that
    // ends the buffer's shared reads
    __device__ __forceinline__ static void refill(const PipeArgs &a, int64_t tile, float2 *buf, uint64_t *bar) {
        if (threadIdx.x == 0) {
            fence_proxy_async_smem();
            issue(a, tile, buf, bar);
        }
    }

    struct Refill {
        static constexpr bool active = true;
        const PipeArgs *a;
        int64_t tile;
        float2 *buf;
        uint64_t *bar;
        __device__ __forceinline__ void operator()() const {
            if (tile >= 0) refill(*a, tile, buf, bar);
        }
    };

    __device__ static void run(const PipeArgs &a) {
        const PassParams &p = a.p;
        // tensor-copy destinations must be 128-byte aligned
        unsigned char *area = dyn_smem_base128();
        float2 *bufs = reinterpret_cast<float2 *>(area + P::TC_BYTES);
        __shared__ __align__(8) uint64_t bars[NBUF];
        const int64_t ntiles = (p.total_lines + C - 1) / C;
        if (threadIdx.x == 0) {
            for (int b = 0; b < NBUF; ++b) mbar_init(&bars[b], 1);
            fence_mbar_init();
        }
        if constexpr (P::NTC > 0) TcUnit<NT, P::TCM_ID, P::E>::setup(p, area);  // ends with a CTA barrier
        __syncthreads();
        if (threadIdx.x == 0)
            for (int b = 0; b < NBUF; ++b) {
                const int64_t t = blockIdx.x + (int64_t)b * gridDim.x;
                if (t < ntiles) issue(a, t, bufs + b * BUF_WORDS, &bars[b]);
            }
        const long long limit = p.spin_limit > 0 ? (long long)p.spin_limit : kMbarSpinLimit;
        for (int64_t k = 0;; ++k) {
            const int64_t tile = blockIdx.x + k * gridDim.x;
            if (tile >= ntiles) break;
            const int b = (int)(k % NBUF);
            const uint32_t parity = (uint32_t)((k / NBUF) & 1);
            if (!mbar_wait_bounded(&bars[b], parity, limit)) {
                if (threadIdx.x == 0 && p.err) atomicExch(p.err, 2);
                // let this CTA's other copies land before the shared memory goes away
                for (int d = 1; d < NBUF; ++d) {
                    const int64_t kk = k + d;
                    if (blockIdx.x + kk * gridDim.x < ntiles)
                        mbar_wait_bounded(&bars[kk % NBUF], (uint32_t)((kk / NBUF) & 1), limit);
                }
                break;
            }
            const int64_t next = tile + (int64_t)NBUF * gridDim.x;
            float2 *buf = bufs + b * BUF_WORDS;
            if constexpr (EARLY) {
                P::run_tile_landed(p, tile, buf, Refill{&a, next < ntiles ? next : -1, buf, &bars[b]}, (uint32_t)k);
            } else {
                P::run_tile_landed(p, tile, buf, NoHook(), (uint32_t)k);
                __syncthreads();  // every shared read of buffer b is done
                if (next < ntiles) refill(a, next, buf, &bars[b]);
            }
        }
        if constexpr (P::NTC > 0) TcUnit<NT, P::TCM_ID, P::E>::teardown(area);
    }
};

template <class P, int NBUF, bool EARLY>
__global__ void __launch_bounds__(P::NT, P::MINB) k_pipe(const __grid_constant__ PipeArgs a) {
    PipeTile<P, NBUF, EARLY>::run(a);
}

// host: encode the tensor map(s) of a four-step pass-1 input (see PipeTile::issue)
bool encode_cols_maps(const PassParams &p, int logl, int lines, int lay, CUtensorMap *tm);

template <class P, int NBUF, bool EARLY>
struct PipeLauncher {
    using PT = PipeTile<P, NBUF, EARLY>;
    static int &grid_cache() {
        static int g = 0;
        return g;
    }
    static cudaError_t prepare() {
        cudaError_t e =
            cudaFuncSetAttribute(k_pipe<P, NBUF, EARLY>, cudaFuncAttributeMaxDynamicSharedMemorySize, PT::SMEM);
        if (e != cudaSuccess) return e;
        int sms = 0, dev = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        const int per_sm = resident_per_sm((const void *)k_pipe<P, NBUF, EARLY>, PT::NT, PT::SMEM,
                                           P::NTC > 0 ? (int)tc_tmem_cols(PT::NT, P::E) : 0);
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        grid_cache() = (per_sm > 0 ? per_sm : 1) * sms;
        return cudaSuccess;
    }
    static cudaError_t launch(const PassParams &p, cudaStream_t st) {
        const int64_t ntiles = (p.total_lines + PT::C - 1) / PT::C;
        if (ntiles <= 0) return cudaSuccess;
        if (grid_cache() == 0) {
            cudaError_t e = prepare();
            if (e != cudaSuccess) return e;
        }
        PipeArgs a;
        memset(&a, 0, sizeof(a));
        a.p = p;
        if constexpr (PT::KIND == KIND_COLS)
            if (!encode_cols_maps(p, P::L == 0 ? 0 : __builtin_ctz(P::L), PT::C, P::LIN_LAYOUT, a.tm))
                return cudaErrorInvalidValue;
        const int grid = (int)(ntiles < grid_cache() ? ntiles : grid_cache());
        k_pipe<P, NBUF, EARLY><<<grid, PT::NT, PT::SMEM, st>>>(a);
        return cudaGetLastError();
    }
};

// `pipe` code of a registry entry: NBUF | 4 * EARLY
constexpr int pipe_code(int nbuf, bool early) { return nbuf | (early ? 4 : 0); }

// registry entry of a pipelined pass kernel
template <int LOGL, int LOGE, int C, int KIND, int LIN, int LOUT, int LOGX, int NBUF, bool EARLY = false,
          int TCM = 0>
constexpr KernelEntry pipe_entry() {
    using P = Pass<LOGL, LOGE, C, KIND, LIN, LOUT, false, LOGX, TCM>;
    using L = PipeLauncher<P, NBUF, EARLY>;
    return KernelEntry{KIND,          LOGL, LOGE, C, LIN, LOUT, P::NT, PipeTile<P, NBUF, EARLY>::SMEM,
                       &L::launch,    &L::prepare, TCM, LOGX, pipe_code(NBUF, EARLY)};
}

}  // namespace fftc

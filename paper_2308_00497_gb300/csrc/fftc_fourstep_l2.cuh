// L2-resident four-step kernel template (the schedule is described in fftc_fourstep_l2.cu).
#pragma once

#include <cstring>

#include "fftc_pass.cuh"

namespace fftc {

struct FsArgs {
    PassParams p1, p2;      // pointers: p1.in / p2.out = user buffers, p1.out / p2.in = slot 0
    unsigned int *ctrl;     // [0] next item, [1 + g] pass-1 done of group g, [1 + G + g] pass-2 done
    int *err;
    long long spin_limit;
    unsigned int wait_bias;  // added to every awaited count: 0, or (test hook) out of reach
    int64_t group_elems;    // GT * n complex elements per group
    int64_t batch, gt;      // transforms in the batch and per group
    int32_t groups, ring, tiles1, tiles2;
};

__device__ __forceinline__ unsigned int fs_ld_acquire(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fs_wait(const FsArgs &a, const unsigned int *cnt, unsigned int target) {
    if (threadIdx.x == 0) {
        long long spins = 0;
        target += a.wait_bias;
        while (fs_ld_acquire(cnt) < target) {
            if (++spins > a.spin_limit) {
                atomicExch(a.err, 1);
                break;
            }
            __nanosleep(64);
        }
    }
    __syncthreads();
}

template <class P1, class P2>
constexpr int fs_min_blocks() {
    constexpr int reg = P1::REG_TARGET > P2::REG_TARGET ? P1::REG_TARGET : P2::REG_TARGET;
    return (65536 / (P1::NT * reg)) > 0 ? (65536 / (P1::NT * reg)) : 1;
}

template <class P1, class P2>
__global__ void __launch_bounds__(P1::NT, fs_min_blocks<P1, P2>()) k_fourstep_l2(const __grid_constant__ FsArgs a) {
    static_assert(P1::NT == P2::NT, "both passes run in the same CTA shape");
    extern __shared__ float2 sm_fs[];
    __shared__ int s_item;
    const int per_block = a.tiles1 + a.tiles2;
    const int total = a.groups * per_block;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(a.ctrl, 1u);
        __syncthreads();
        const int w = s_item;
        if (w >= total) break;
        // decode: block b holds P1(b) (b < G) then P2(b - 1) (b >= 1)
        int b, r;
        if (w < a.tiles1) {
            b = 0;
            r = w;
        } else {
            b = 1 + (w - a.tiles1) / per_block;
            r = (w - a.tiles1) % per_block;
        }
        const bool pass1 = (b < a.groups) && (r < a.tiles1);
        const int g = pass1 ? b : b - 1;
        const int tile = pass1 ? r : (b < a.groups ? r - a.tiles1 : r);
        const int slot = g % a.ring;
        const int64_t gt = min(a.gt, a.batch - (int64_t)g * a.gt);  // transforms in this group
        const int64_t uoff = (int64_t)g * a.group_elems;             // complex offset in user buffers
        const int64_t woff = (int64_t)slot * a.group_elems;          // complex offset in the workspace
        if (pass1) {
            if (g >= a.ring) fs_wait(a, a.ctrl + 1 + a.groups + (g - a.ring), (unsigned)a.tiles2);
            PassParams p = a.p1;
            p.in = p.in + uoff * (p.in_plane ? 1 : 2);  // split planes are indexed per element
            p.out = p.out + 2 * woff;
            p.total_lines = gt << p.log_lpt;
            P1::run_tile(p, tile, sm_fs);
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) atomicAdd(a.ctrl + 1 + g, 1u);
        } else {
            fs_wait(a, a.ctrl + 1 + g, (unsigned)a.tiles1);
            PassParams p = a.p2;
            p.in = p.in + 2 * woff;
            p.out = p.out + uoff * (p.out_plane ? 1 : 2);
            p.total_lines = gt << p.log_lpt;
            P2::run_tile(p, tile, sm_fs);
            __syncthreads();  // every read of the tile's workspace rows has completed
            {
                // rows [tile * C, tile * C + C) of the group: C * K consecutive elements
                const int64_t first = (int64_t)tile * P2::NT / P2::TPL;  // = tile * C lines
                const int64_t lines = min((int64_t)(P2::NT / P2::TPL), (gt << a.p2.log_lpt) - first);
                if (lines > 0) {
                    const char *base = reinterpret_cast<const char *>(a.p2.in + 2 * (woff + first * P2::L));
                    const int64_t nbytes = lines * P2::L * (int64_t)sizeof(float2);
                    for (int64_t o = (int64_t)threadIdx.x * 128; o < nbytes; o += (int64_t)P2::NT * 128)
                        asm volatile("discard.global.L2 [%0], 128;" ::"l"(base + o) : "memory");
                }
            }
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) atomicAdd(a.ctrl + 1 + a.groups + g, 1u);
        }
        __syncthreads();  // s_item and shared memory are reused by the next item
    }
}

// ---------------------------------------------------------------------------
// instances: one per n = 2^14 .. 2^20 and layout, both passes with the same CTA size
// ---------------------------------------------------------------------------
struct FsEntry {
    int logn, logm, e1, c1, e2, c2, lay;
    void (*kernel)(FsArgs);
    int threads, smem;
};

template <int LOGM, int E1, int C1, int LOGK, int E2, int C2, int LAY>
constexpr FsEntry fs_entry() {
    using P1 = Pass<LOGM, E1, C1, KIND_COLS, LAY, LAYOUT_IL, false, LOGK>;
    using P2 = Pass<LOGK, E2, C2, KIND_ROWST, LAYOUT_IL, LAY, false, LOGM>;
    return FsEntry{LOGM + LOGK, LOGM, E1, C1, E2, C2, LAY, &k_fourstep_l2<P1, P2>, P1::NT,
                   P1::SMEM > P2::SMEM ? P1::SMEM : P2::SMEM};
}

}  // namespace fftc

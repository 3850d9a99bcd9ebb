// L2-resident four-step transform: both passes of Eq. 1 applied at the memory level
// (n = M K) run in ONE persistent launch, group by group, so that the pass-1 output
// of a group is still in L2 when pass 2 reads it. Only the input read (pass 1) and
// the output write (pass 2) reach HBM: 16 B per element instead of 32.
//
// The batch is cut into groups of GT transforms (about FFTC_L2_GROUP_MB of data).
// Group g's workspace is slot g mod W of a ring of W >= 2 slots. Work items, taken in
// order with one atomic add:
//   P1(0) | P1(1) P2(0) | P1(2) P2(1) | ... | P2(G-1)
// A pass-2 tile of group g waits until every pass-1 tile of g has signalled; a pass-1
// tile of group g >= W waits until every pass-2 tile of group g - W (the previous user
// of its slot) has signalled. Every awaited item precedes the waiting one in the order
// and never waits on a later item, so with W >= 2 the waits always end; each is a
// bounded spin that sets the plan's error word if it gives up. After a pass-2 tile has
// read its workspace rows it discards those L2 lines (discard.global.L2), so the dirty
// workspace is never written back to HBM; pass 1 of the slot's next group overwrites
// every discarded word before it is read again.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "fftc_pass.cuh"
#include "fftc_plan.h"

namespace fftc {

struct FsArgs {
    PassParams p1, p2;      // pointers: p1.in / p2.out = user buffers, p1.out / p2.in = slot 0
    unsigned int *ctrl;     // [0] next item, [1 + g] pass-1 done of group g, [1 + G + g] pass-2 done
    int *err;
    long long spin_limit;
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

#define FS2(LOGM, E1, C1, LOGK, E2, C2) \
    fs_entry<LOGM, E1, C1, LOGK, E2, C2, LAYOUT_IL>(), fs_entry<LOGM, E1, C1, LOGK, E2, C2, LAYOUT_SPLIT>()

static const FsEntry kFsTable[] = {
    FS2(7, 4, 16, 7, 4, 16),   // 2^14: 128 threads
    FS2(7, 4, 16, 8, 5, 16),   // 2^15: 128
    FS2(8, 4, 16, 8, 4, 16),   // 2^16: 256
    FS2(8, 4, 16, 9, 5, 16),   // 2^17: 256
    FS2(9, 5, 16, 9, 5, 16),   // 2^18: 256
    FS2(9, 5, 16, 10, 5, 8),   // 2^19: 256
    FS2(10, 5, 8, 10, 5, 8),   // 2^20: 256
};

static const FsEntry *find_fs(int logn, int lay) {
    for (const FsEntry &e : kFsTable)
        if (e.logn == logn && e.lay == lay) return &e;
    return nullptr;
}

struct FsState {
    const FsEntry *e = nullptr;
    FsArgs args{};
    unsigned int *ctrl = nullptr;
    int n_ctrl = 0;
    int grid = 0;
};

static int env_int_fs(const char *name, int dflt) {
    const char *v = getenv(name);
    return (v && *v) ? atoi(v) : dflt;
}

// Off by default until it beats the two-launch path (FFTC_L2_RESIDENT=1 enables it).
bool fs_available(int logn, int lay) { return env_int_fs("FFTC_L2_RESIDENT", 0) != 0 && find_fs(logn, lay) != nullptr; }

void fs_free(fftc_plan_s *p) {
    delete p->fs;
    p->fs = nullptr;
}

// Build the L2-resident executor of a four-step FP32 plan: workspace ring, counters,
// stage tables and the inter-pass diagonal D (already in p->tw2_full).
fftc_status fs_build(fftc_plan_s *p) {
    const int lay = p->layout == FFTC_LAYOUT_SPLIT ? LAYOUT_SPLIT : LAYOUT_IL;
    const FsEntry *e = find_fs(p->logn, lay);
    if (!e) return FFTC_ERR_UNSUPPORTED_SIZE;
    // stage tables of this executor's own radix choice
    const float2 *tw1 = nullptr, *tw2 = nullptr;
    {
        std::vector<float2> t;
        void *dt = nullptr;
        stage_twiddles(e->logm, e->e1, t);
        if (plan_upload(p, t.data(), t.size() * sizeof(float2), &dt) != cudaSuccess) return FFTC_ERR_ALLOC;
        tw1 = (const float2 *)dt;
        stage_twiddles(p->logn - e->logm, e->e2, t);
        if (plan_upload(p, t.data(), t.size() * sizeof(float2), &dt) != cudaSuccess) return FFTC_ERR_ALLOC;
        tw2 = (const float2 *)dt;
    }
    FsState *s = new (std::nothrow) FsState();
    if (!s) return FFTC_ERR_ALLOC;
    p->fs = s;
    s->e = e;
    const int64_t n = p->n, B = p->batch;
    const int logm = e->logm, logk = p->logn - logm;
    const int64_t M = int64_t(1) << logm, K = int64_t(1) << logk;
    const int64_t group_bytes = (int64_t)env_int_fs("FFTC_L2_GROUP_MB", 16) << 20;
    int64_t gt = std::max<int64_t>(1, group_bytes / (n * 8));
    gt = std::min<int64_t>(gt, std::max<int64_t>(B, 1));
    const int ring = std::max(2, env_int_fs("FFTC_L2_RING", 3));
    const int64_t groups = (B + gt - 1) / gt;
    if (groups > (1 << 24)) return FFTC_ERR_UNSUPPORTED_SIZE;
    void *d = nullptr;
    if (plan_alloc(p, (size_t)(ring * gt * n) * sizeof(float2), &d) != cudaSuccess) return FFTC_ERR_ALLOC;
    float2 *ws = (float2 *)d;
    s->n_ctrl = 1 + 2 * (int)groups;
    if (plan_alloc(p, (size_t)s->n_ctrl * sizeof(unsigned int), &d) != cudaSuccess) return FFTC_ERR_ALLOC;
    s->ctrl = (unsigned int *)d;

    FsArgs &a = s->args;
    const int64_t plane = lay == LAYOUT_SPLIT ? n * B : 0;
    PassParams &p1 = a.p1;
    memset(&p1, 0, sizeof(p1));
    p1.in_plane = plane;
    p1.log_lpt = logk;
    p1.in_tr = p1.out_tr = n;
    p1.in_line = p1.out_line = 1;
    p1.in_elem = p1.out_elem = K;
    p1.tw = tw1;
    p1.tw2_full = p->tw2_full;
    p1.tw2_lo = p->tw2_lo;
    p1.tw2_hi = p->tw2_hi;
    p1.log_n2 = p->logn;
    p1.tw2_lo_bits = p->tw2_lo_bits;
    p1.out = (float *)ws;
    PassParams &p2 = a.p2;
    memset(&p2, 0, sizeof(p2));
    p2.out_plane = plane;
    p2.log_lpt = logm;
    p2.in_tr = p2.out_tr = n;
    p2.in_line = K;
    p2.in_elem = 1;
    p2.out_line = 1;
    p2.out_elem = M;
    p2.post_line_mul = 1;
    p2.post_elem_mul = M;
    p2.tw = tw2;
    p2.in = (const float *)ws;
    a.ctrl = s->ctrl;
    a.err = p->d_err;
    a.spin_limit = (long long)env_int_fs("FFTC_SPIN_LIMIT", 20000000);
    a.group_elems = gt * n;
    a.batch = B;
    a.gt = gt;
    a.groups = (int32_t)groups;
    a.ring = ring;
    a.tiles1 = (int32_t)((gt * K) / e->c1);
    a.tiles2 = (int32_t)((gt * M) / e->c2);

    if (e->smem > 48 * 1024 &&
        cudaFuncSetAttribute(e->kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, e->smem) != cudaSuccess)
        return FFTC_ERR_CUDA;
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, e->kernel, e->threads, e->smem) != cudaSuccess)
        return FFTC_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) return FFTC_ERR_CUDA;
    s->grid = std::max(1, per_sm) * sms;
    return FFTC_OK;
}

fftc_status fs_run(fftc_plan_s *p, const void *in, void *out, const float *post_h, float post_scale, cudaStream_t st) {
    FsState *s = p->fs;
    FsArgs a = s->args;
    const int inv = p->direction == FFTC_INVERSE ? 1 : 0;
    a.p1.in = (const float *)in;
    a.p1.conj_in = inv;
    a.p2.out = (float *)out;
    a.p2.conj_out = inv;
    a.p2.post_h = post_h;
    a.p2.post_scale = post_scale;
    if (cudaMemsetAsync(s->ctrl, 0, (size_t)s->n_ctrl * sizeof(unsigned int), st) != cudaSuccess) return FFTC_ERR_CUDA;
    void *kargs[] = {&a};
    if (cudaLaunchKernel((const void *)s->e->kernel, dim3(s->grid), dim3(s->e->threads), kargs, (size_t)s->e->smem,
                         st) != cudaSuccess)
        return FFTC_ERR_CUDA;
    return FFTC_OK;
}

}  // namespace fftc

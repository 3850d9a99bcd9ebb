// Uneven batches: many transforms of different power-of-two lengths in ONE persistent
// kernel launch, replayed from a CUDA graph built when the plan is created.
//
// Every transform is cut into CTA tiles of a fused Stockham pass (fftc_pass.cuh):
//   n <= 2^12 (by default): single-pass tiles; the transforms of one length form a
//             "class" whose rows are gathered by offset (indexed lines), C rows a tile;
//   n >= 2^13: the four-step split of Eq. 1 (n = M * K): pass-1 column tiles write a
//             per-transform workspace, pass-2 row tiles read it back.
// A work list orders the tiles (pass-1 tiles of the largest transforms first, then the
// single-pass tiles from large to small, then the pass-2 tiles); CTAs take the next item
// with one atomic add. A pass-2 tile first waits (bounded spin, thread 0, acquire load)
// until every pass-1 tile of its transform has signalled completion; pass-1 tiles never
// wait, and any pass-1 tile a pass-2 tile depends on was taken earlier by a running CTA,
// so the waits always end. A wait that exceeds its iteration limit sets the plan's error
// word and the tile proceeds (fftc_plan_check then reports FFTC_ERR_TIMEOUT).
// All branches run 256-thread CTAs with E <= 16 (4 CTAs per SM).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fftc.h"
#include "fftc_pass.cuh"
#include "fftc_plan.h"

namespace fftc {

// (id, LOGL, LOGE, C, KIND, IDX, LOGX): every branch has C * 2^(LOGL - LOGE) = 256
// threads; the four-step branches carry their element stride 2^LOGX at compile time
// (one pair per split n = M K of the classes 2^13 .. 2^16). Branches 19..34 are the "half"
// variants: half the elements per thread, so twice the threads per line, half the lines
// per tile and one more radix stage; branches 35.. the "wide" four-step variants: 16
// elements per thread whatever the line length, so short lines (64, 128) come in tiles of
// 4096 elements (64 or 32 lines) instead of 16 lines (the autotuner's tile-shape /
// stages-per-pass choice).
#define FFTC_UNEVEN_BRANCHES(X)                \
    X(0, 6, 4, 64, KIND_ROWS, true, 0)         \
    X(1, 7, 4, 32, KIND_ROWS, true, 0)         \
    X(2, 8, 4, 16, KIND_ROWS, true, 0)         \
    X(3, 9, 4, 8, KIND_ROWS, true, 0)          \
    X(4, 10, 4, 4, KIND_ROWS, true, 0)         \
    X(5, 11, 4, 2, KIND_ROWS, true, 0)         \
    X(6, 12, 4, 1, KIND_ROWS, true, 0)         \
    X(7, 6, 2, 16, KIND_COLS, false, 7)        \
    X(8, 7, 3, 16, KIND_COLS, false, 6)        \
    X(9, 7, 3, 16, KIND_COLS, false, 7)        \
    X(10, 7, 3, 16, KIND_COLS, false, 8)       \
    X(11, 8, 4, 16, KIND_COLS, false, 7)       \
    X(12, 8, 4, 16, KIND_COLS, false, 8)       \
    X(13, 7, 3, 16, KIND_ROWST, false, 6)      \
    X(14, 6, 2, 16, KIND_ROWST, false, 7)      \
    X(15, 7, 3, 16, KIND_ROWST, false, 7)      \
    X(16, 8, 4, 16, KIND_ROWST, false, 7)      \
    X(17, 7, 3, 16, KIND_ROWST, false, 8)      \
    X(18, 8, 4, 16, KIND_ROWST, false, 8)      \
    X(19, 6, 3, 32, KIND_ROWS, true, 0)        \
    X(20, 7, 3, 16, KIND_ROWS, true, 0)        \
    X(21, 8, 3, 8, KIND_ROWS, true, 0)         \
    X(22, 9, 3, 4, KIND_ROWS, true, 0)         \
    X(23, 10, 3, 2, KIND_ROWS, true, 0)        \
    X(24, 11, 3, 1, KIND_ROWS, true, 0)        \
    X(25, 7, 2, 8, KIND_COLS, false, 6)        \
    X(26, 7, 2, 8, KIND_COLS, false, 7)        \
    X(27, 7, 2, 8, KIND_COLS, false, 8)        \
    X(28, 8, 3, 8, KIND_COLS, false, 7)        \
    X(29, 8, 3, 8, KIND_COLS, false, 8)        \
    X(30, 7, 2, 8, KIND_ROWST, false, 6)       \
    X(31, 7, 2, 8, KIND_ROWST, false, 7)       \
    X(32, 7, 2, 8, KIND_ROWST, false, 8)       \
    X(33, 8, 3, 8, KIND_ROWST, false, 7)       \
    X(34, 8, 3, 8, KIND_ROWST, false, 8)       \
    X(35, 6, 4, 64, KIND_COLS, false, 7)       \
    X(36, 6, 4, 64, KIND_COLS, false, 8)       \
    X(37, 7, 4, 32, KIND_COLS, false, 6)       \
    X(38, 7, 4, 32, KIND_COLS, false, 7)       \
    X(39, 7, 4, 32, KIND_COLS, false, 8)       \
    X(40, 8, 4, 16, KIND_COLS, false, 6)       \
    X(41, 6, 4, 64, KIND_ROWST, false, 7)      \
    X(42, 6, 4, 64, KIND_ROWST, false, 8)      \
    X(43, 7, 4, 32, KIND_ROWST, false, 6)      \
    X(44, 7, 4, 32, KIND_ROWST, false, 7)      \
    X(45, 7, 4, 32, KIND_ROWST, false, 8)      \
    X(46, 8, 4, 16, KIND_ROWST, false, 6)

#define FFTC_BRANCH_TYPE(ID, LOGL, LOGE, C, KIND, IDX, LOGX) \
    Pass<LOGL, LOGE, C, KIND, LAYOUT_IL, LAYOUT_IL, IDX, LOGX>

struct BranchInfo {
    int logl, loge, lines, kind, logx, smem;
};
#define FFTC_BRANCH_INFO(ID, LOGL, LOGE, C, KIND, IDX, LOGX) \
    BranchInfo{LOGL, LOGE, C, KIND, LOGX, FFTC_BRANCH_TYPE(ID, LOGL, LOGE, C, KIND, IDX, LOGX)::SMEM},
static const BranchInfo kBranches[] = {FFTC_UNEVEN_BRANCHES(FFTC_BRANCH_INFO)};
static const int kNumBranches = sizeof(kBranches) / sizeof(kBranches[0]);

#define FFTC_BRANCH_CHECK(ID, LOGL, LOGE, C, KIND, IDX, LOGX)                             \
    static_assert(FFTC_BRANCH_TYPE(ID, LOGL, LOGE, C, KIND, IDX, LOGX)::NT == 256,        \
                  "uneven branches use 256 threads");
FFTC_UNEVEN_BRANCHES(FFTC_BRANCH_CHECK)

static constexpr int kUnevenThreads = 256;
// CTAs per SM the kernel is compiled for (64 registers a thread at 4): measured on the
// 4096-row workload, 3 (80 registers) 0.350 ms, 4 0.312 ms, 5 (48 registers, spilling)
// 0.328 ms
static constexpr int kUnevenCtasPerSm = 4;

struct WorkItem {
    int32_t branch, param, tile;
    int32_t wait_idx, wait_target;  // wait until done[wait_idx] >= wait_target (-1: none)
    int32_t signal_idx;             // after the tile: done[signal_idx] += 1 (-1: none)
};

struct PersArgs {
    const WorkItem *items;
    const PassParams *params;
    const int8_t *branch_logl, *branch_lines, *branch_kind;  // per branch: log2 L, lines per tile, kind
    unsigned int *ctrl;  // ctrl[0] = next work item, ctrl[1 + i] = done counter i
    const float *in;
    float *out;
    int *err;
    long long spin_limit;
    int32_t n_items;
    int32_t pf_ahead;  // a CTA that takes item i asks L2 for the input of item i + pf_ahead (0 = off)
};

// Ask L2 for the HBM input of a work item (single-pass rows or a four-step column band),
// one prefetch per 32-byte sector; the CTA that takes the item about one wave later then
// finds it in L2. Pass-2 tiles read the workspace, which is still in L2: nothing to fetch.
__device__ __forceinline__ void prefetch_item(const PersArgs &a, const WorkItem &it) {
    const int kind = a.branch_kind[it.branch];
    if (kind == KIND_ROWST) return;
    const PassParams &p = a.params[it.param];
    const char *in = reinterpret_cast<const char *>(p.in);
    if (p.in_user) in = reinterpret_cast<const char *>(a.in) + (intptr_t)p.in;
    const int L = 1 << a.branch_logl[it.branch], C = a.branch_lines[it.branch];
    const int64_t g0 = (int64_t)it.tile * C;
    if (kind == KIND_ROWS) {  // C indexed lines of L contiguous elements
        const int spl = L * 8 / 32;
        for (int i = threadIdx.x; i < C * spl; i += blockDim.x) {
            const int64_t g = g0 + i / spl;
            if (g < p.total_lines) prefetch_l2(in + __ldg(p.line_off + g) * 8 + (i % spl) * 32);
        }
    } else {  // L rows of C adjacent columns at element stride in_elem
        const int spr = (C * 8 + 31) / 32;
        const int64_t base = (g0 >> p.log_lpt) * p.in_tr + (g0 & ((int64_t(1) << p.log_lpt) - 1)) * p.in_line;
        for (int i = threadIdx.x; i < L * spr; i += blockDim.x)
            prefetch_l2(in + (base + (int64_t)(i / spr) * p.in_elem) * 8 + (i % spr) * 32);
    }
}

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Drop the L2 lines of workspace rows a pass-2 tile has finished reading (`elems`
// complex elements from `ws`): the workspace is never read again in this launch, so its
// dirty lines need not be written back to HBM. Called after a CTA barrier that follows
// the tile: every load of the tile has returned by then (each thread consumed its loads
// before the tile's first exchange barrier).
__device__ __forceinline__ void discard_rows(const float *ws, int elems) {
    const char *base = reinterpret_cast<const char *>(ws);
    for (int o = threadIdx.x * 128; o < elems * 8; o += kUnevenThreads * 128)
        asm volatile("discard.global.L2 [%0], 128;" ::"l"(base + o) : "memory");
}

template <int MINB>
__global__ void __launch_bounds__(kUnevenThreads, MINB) k_uneven(const __grid_constant__ PersArgs a) {
    extern __shared__ float2 sm_pers[];
    __shared__ int s_idx[2];  // the item in hand and the item claimed after it
    if (threadIdx.x == 0) s_idx[0] = (int)atomicAdd(a.ctrl, 1u);
    __syncthreads();
    for (int cur = 0;; cur ^= 1) {
        const int idx = s_idx[cur];
        if (idx >= a.n_items) break;
        // Claim the next item now, so the CTA goes straight on to it when this one ends.
        // Claims follow the list order, so the earliest unfinished item is always the
        // item in hand of some CTA, and every item a pass-2 tile waits for comes before
        // it in the list: the waits still end.
        if (threadIdx.x == 0) s_idx[cur ^ 1] = (int)atomicAdd(a.ctrl, 1u);
        const WorkItem it = a.items[idx];
        if (a.pf_ahead > 0 && idx + a.pf_ahead < a.n_items) prefetch_item(a, a.items[idx + a.pf_ahead]);
        if (it.wait_idx >= 0) {
            if (threadIdx.x == 0) {
                long long spins = 0;
                while (ld_acquire_gpu(a.ctrl + 1 + it.wait_idx) < (unsigned)it.wait_target) {
                    if (++spins > a.spin_limit) {
                        atomicExch(a.err, 1);
                        break;
                    }
                    __nanosleep(128);
                }
            }
            __syncthreads();  // the acquire by thread 0 orders the tile's workspace loads
        }
        PassParams p = a.params[it.param];
        if (p.in_user) p.in = reinterpret_cast<const float *>(reinterpret_cast<const char *>(a.in) + (intptr_t)p.in);
        if (p.out_user) p.out = reinterpret_cast<float *>(reinterpret_cast<char *>(a.out) + (intptr_t)p.out);
        const float *ws_done = nullptr;
        int ws_elems = 0;
        switch (it.branch) {
#define FFTC_BRANCH_CASE(ID, LOGL, LOGE, C, KIND, IDX, LOGX)                                 \
    case ID:                                                                                 \
        FFTC_BRANCH_TYPE(ID, LOGL, LOGE, C, KIND, IDX, LOGX)::run_tile(p, it.tile, sm_pers);  \
        if (KIND == KIND_ROWST) {                                                            \
            ws_done = p.in + 2 * (int64_t)it.tile * C * (1 << LOGL);                         \
            ws_elems = C << LOGL;                                                            \
        }                                                                                    \
        break;
            FFTC_UNEVEN_BRANCHES(FFTC_BRANCH_CASE)
            default: break;
        }
        // One barrier ends the item: every thread's stores of the tile are issued, its
        // shared memory may be reused, and the claim of the next item is visible.
        __syncthreads();
        if (ws_elems) discard_rows(ws_done, ws_elems);
        if (it.signal_idx >= 0 && threadIdx.x == 0) {
            // after the barrier, thread 0's device-scope fence orders the whole CTA's stores
            // of the tile before the counter increment that releases its pass-2 tiles
            __threadfence();
            atomicAdd(a.ctrl + 1 + it.signal_idx, 1u);
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct UnevenState {
    std::vector<WorkItem> items;
    std::vector<PassParams> params;
    WorkItem *d_items = nullptr;
    PassParams *d_params = nullptr;
    int8_t *d_branch = nullptr;  // per branch: log2 L, lines per tile, kind (3 x kNumBranches)
    unsigned int *d_ctrl = nullptr;
    int n_ctrl = 0;
    int grid = 0, smem = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t knode = nullptr;
    void *kfunc = nullptr;  // the k_uneven instance
    PersArgs args{};
    int max_logn = 0;
    int64_t total_elems = 0;
};

static int find_branch(int kind, int logl, int loge, int lines, int logx = 0) {
    for (int i = 0; i < kNumBranches; ++i)
        if (kBranches[i].kind == kind && kBranches[i].logl == logl && kBranches[i].loge == loge &&
            kBranches[i].lines == lines && kBranches[i].logx == logx)
            return i;
    return -1;
}

// Configuration of one length class: single pass (logm = 0) or four-step (logm > 0), with
// the default elements per thread (ev = 0), half of them (ev = 1: twice the threads per
// line, half the lines per tile, one more radix stage) or, four-step only, 16 elements per
// thread on every line length (ev = 2: 4096-element tiles). Passed around as one int code.
struct ClassCfg {
    int logm = 0;  // four-step split n = 2^logm * 2^(logn - logm); 0 = single pass
    int ev = 0;
    static ClassCfg decode(int code) {
        ClassCfg c;
        c.logm = code & 0xff;
        c.ev = code >> 8;
        return c;
    }
    int code() const { return logm | (ev << 8); }
};

static int env_int(const char *name, int dflt) {
    const char *v = getenv(name);
    return (v && *v) ? atoi(v) : dflt;
}


static int rows_branch(int logn, int ev) {
    if (ev > 1) return -1;
    const int loge = 4 - ev;
    return logn > loge ? find_branch(KIND_ROWS, logn, loge, 256 >> (logn - loge)) : -1;
}
static int cols_branch(int logm, int logk, int ev) {
    if (ev == 2) return find_branch(KIND_COLS, logm, 4, 256 >> (logm - 4), logk);
    return find_branch(KIND_COLS, logm, logm - 4 - ev, 16 >> ev, logk);
}
static int rowst_branch(int logk, int logm, int ev) {
    if (ev == 2) return find_branch(KIND_ROWST, logk, 4, 256 >> (logk - 4), logm);
    return find_branch(KIND_ROWST, logk, logk - 4 - ev, 16 >> ev, logm);
}

static bool class_supported(int logn, const ClassCfg &c) {
    if (c.logm == 0) return rows_branch(logn, c.ev) >= 0;
    const int logk = logn - c.logm;
    return cols_branch(c.logm, logk, c.ev) >= 0 && rowst_branch(logk, c.logm, c.ev) >= 0;
}

int uneven_max_logn(const fftc_plan_s *p) { return p->uneven ? p->uneven->max_logn : 0; }

void uneven_free(fftc_plan_s *p) {
    UnevenState *u = p->uneven;
    if (!u) return;
    if (u->exec) cudaGraphExecDestroy(u->exec);
    if (u->graph) cudaGraphDestroy(u->graph);
    delete u;
    p->uneven = nullptr;
}

static cudaError_t build_graph(UnevenState *u, int *d_err, cudaStream_t st) {
    (void)st;
    cudaError_t e = cudaGraphCreate(&u->graph, 0);
    if (e != cudaSuccess) return e;
    cudaGraphNode_t mnode;
    cudaMemsetParams mp{};
    mp.dst = u->d_ctrl;
    mp.value = 0;
    mp.elementSize = 4;
    mp.width = (size_t)u->n_ctrl;
    mp.height = 1;
    mp.pitch = 0;
    if ((e = cudaGraphAddMemsetNode(&mnode, u->graph, nullptr, 0, &mp)) != cudaSuccess) return e;
    u->args.items = u->d_items;
    u->args.params = u->d_params;
    u->args.branch_logl = u->d_branch;
    u->args.branch_lines = u->d_branch + kNumBranches;
    u->args.branch_kind = u->d_branch + 2 * kNumBranches;
    u->args.ctrl = u->d_ctrl;
    u->args.err = d_err;
    u->args.n_items = (int32_t)u->items.size();
    u->args.in = nullptr;
    u->args.out = nullptr;
    void *kargs[] = {&u->args};
    cudaKernelNodeParams kp{};
    kp.func = u->kfunc;
    kp.gridDim = dim3(u->grid);
    kp.blockDim = dim3(kUnevenThreads);
    kp.sharedMemBytes = u->smem;
    kp.kernelParams = kargs;
    if ((e = cudaGraphAddKernelNode(&u->knode, u->graph, &mnode, 1, &kp)) != cudaSuccess) return e;
    return cudaGraphInstantiate(&u->exec, u->graph, 0);
}

fftc_status uneven_run(fftc_plan_s *p, const void *in, void *out, cudaStream_t st) {
    UnevenState *u = p->uneven;
    if (u->args.in != in || u->args.out != out) {
        u->args.in = (const float *)in;
        u->args.out = (float *)out;
        void *kargs[] = {&u->args};
        cudaKernelNodeParams kp{};
        kp.func = u->kfunc;
        kp.gridDim = dim3(u->grid);
        kp.blockDim = dim3(kUnevenThreads);
        kp.sharedMemBytes = u->smem;
        kp.kernelParams = kargs;
        if (cudaGraphExecKernelNodeSetParams(u->exec, u->knode, &kp) != cudaSuccess) return FFTC_ERR_CUDA;
    }
    if (cudaGraphLaunch(u->exec, st) != cudaSuccess) return FFTC_ERR_CUDA;
    return FFTC_OK;
}

typedef int (*ClassChoice)(int logn, void *ctx);

static fftc_status build_state(fftc_plan_s *p, int64_t count, const int64_t *n, const int8_t *dir,
                               const int64_t *off, ClassChoice choose, void *ctx) {
    UnevenState *u = new (std::nothrow) UnevenState();
    if (!u) return FFTC_ERR_ALLOC;
    p->uneven = u;

    // validate and find the extent of the buffers
    std::vector<int64_t> order((size_t)count);
    int64_t total = 0;
    for (int64_t i = 0; i < count; ++i) {
        if (n[i] < 64 || n[i] > (int64_t(1) << 16) || (n[i] & (n[i] - 1))) return FFTC_ERR_UNSUPPORTED_SIZE;
        if (dir[i] != -1 && dir[i] != 1) return FFTC_ERR_INVALID_VALUE;
        if (off[i] < 0) return FFTC_ERR_INVALID_VALUE;
        order[(size_t)i] = i;
        total = std::max(total, off[i] + n[i]);
    }
    std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return off[a] < off[b]; });
    for (size_t k = 1; k < order.size(); ++k)
        if (off[order[k - 1]] + n[order[k - 1]] > off[order[k]]) return FFTC_ERR_INVALID_VALUE;  // overlap
    u->total_elems = total;
    p->total_elems = total;

    // classes by length
    std::map<int, std::vector<int64_t>> by_log;
    for (int64_t i = 0; i < count; ++i) {
        int lg = 0;
        while ((int64_t(1) << lg) < n[i]) ++lg;
        by_log[lg].push_back(i);
        u->max_logn = std::max(u->max_logn, lg);
    }

    // device tables: stage twiddles per (L, E), inter-pass tables per four-step length
    std::map<std::pair<int, int>, float2 *> stage_tab;
    auto stage_table = [&](int logl, int loge, float2 **out) -> fftc_status {
        auto key = std::make_pair(logl, loge);
        auto it = stage_tab.find(key);
        if (it != stage_tab.end()) {
            *out = it->second;
            return FFTC_OK;
        }
        std::vector<float2> tw;
        stage_twiddles(logl, loge, tw);
        void *d = nullptr;
        if (plan_upload(p, tw.data(), tw.size() * sizeof(float2), &d) != cudaSuccess) return FFTC_ERR_ALLOC;
        stage_tab[key] = (float2 *)d;
        *out = (float2 *)d;
        return FFTC_OK;
    };

    // workspace for the four-step transforms
    int64_t ws_elems = 0;
    std::map<int, ClassCfg> cfg;
    for (auto &kv : by_log) {
        const int code = choose(kv.first, ctx);
        if (code < 0) return FFTC_ERR_UNSUPPORTED_SIZE;
        const ClassCfg c = ClassCfg::decode(code);
        if (!class_supported(kv.first, c)) return FFTC_ERR_UNSUPPORTED_SIZE;
        cfg[kv.first] = c;
        if (c.logm) ws_elems += (int64_t(1) << kv.first) * (int64_t)kv.second.size();
    }
    void *d = nullptr;
    float2 *ws = nullptr;
    if (ws_elems) {
        if (plan_alloc(p, (size_t)ws_elems * sizeof(float2), &d) != cudaSuccess) return FFTC_ERR_ALLOC;
        ws = (float2 *)d;
    }

    // Work items. The pass-2 tiles of a four-step transform are queued once FFTC_UNEVEN_LAG_MB
    // (default 24) of later pass-1 input has been queued behind its pass-1 tiles: late enough
    // that they rarely wait, early enough that the workspace is still in L2. Single-pass tiles
    // follow, then the pass-2 tiles still pending.
    std::vector<WorkItem> p1, p0, p2;
    struct Pending {
        double release;
        std::vector<WorkItem> items;
    };
    std::vector<Pending> pend;
    size_t pend_head = 0;
    double queued_bytes = 0.0;
    const double lag_bytes = (double)env_int("FFTC_UNEVEN_LAG_MB", 24) * (1 << 20);
    int n_done = 0;
    int64_t ws_off = 0;
    for (auto it = by_log.rbegin(); it != by_log.rend(); ++it) {
        const int logn = it->first;
        const std::vector<int64_t> &ids = it->second;
        const ClassCfg &c = cfg[logn];
        const int64_t nn = int64_t(1) << logn;
        if (c.logm == 0) {
            const int b = rows_branch(logn, c.ev);
            const BranchInfo &bi = kBranches[b];
            std::vector<int64_t> loff(ids.size());
            std::vector<int8_t> lconj(ids.size());
            for (size_t k = 0; k < ids.size(); ++k) {
                loff[k] = off[ids[k]];
                lconj[k] = dir[ids[k]] == 1 ? 1 : 0;
            }
            if (plan_upload(p, loff.data(), loff.size() * sizeof(int64_t), &d) != cudaSuccess) return FFTC_ERR_ALLOC;
            const int64_t *d_off = (const int64_t *)d;
            if (plan_upload(p, lconj.data(), lconj.size(), &d) != cudaSuccess) return FFTC_ERR_ALLOC;
            const int8_t *d_conj = (const int8_t *)d;
            PassParams q{};
            float2 *tw = nullptr;
            fftc_status s = stage_table(logn, bi.loge, &tw);
            if (s != FFTC_OK) return s;
            q.tw = tw;
            q.total_lines = (int64_t)ids.size();
            q.in_elem = q.out_elem = 1;
            q.line_off = d_off;
            q.line_conj = d_conj;
            q.in_user = q.out_user = 1;
            q.in = nullptr;  // byte offset 0 into the user buffers
            q.out = nullptr;
            const int pi = (int)u->params.size();
            u->params.push_back(q);
            const int64_t tiles = ((int64_t)ids.size() + bi.lines - 1) / bi.lines;
            for (int64_t t = 0; t < tiles; ++t) p0.push_back(WorkItem{b, pi, (int32_t)t, -1, 0, -1});
        } else {
            const int logm = c.logm, logk = logn - logm;
            const int64_t M = int64_t(1) << logm, K = int64_t(1) << logk;
            const int b1 = cols_branch(logm, logk, c.ev), b2 = rowst_branch(logk, logm, c.ev);
            float2 *tw1 = nullptr, *tw2 = nullptr;
            fftc_status s = stage_table(logm, kBranches[b1].loge, &tw1);
            if (s != FFTC_OK) return s;
            if ((s = stage_table(logk, kBranches[b2].loge, &tw2)) != FFTC_OK) return s;
            // inter-pass tables of this length
            const int lob = (logn + 1) / 2;
            const int64_t nlo = int64_t(1) << lob, nhi = nn >> lob;
            std::vector<float2> lo(nlo), hi(nhi);
            for (int64_t m = 0; m < nlo; ++m) {
                double cc, ss;
                unit_root(m, nn, &cc, &ss);
                lo[m] = make_float2((float)cc, (float)-ss);
            }
            for (int64_t m = 0; m < nhi; ++m) {
                double cc, ss;
                unit_root(m * nlo, nn, &cc, &ss);
                hi[m] = make_float2((float)cc, (float)-ss);
            }
            if (plan_upload(p, lo.data(), lo.size() * sizeof(float2), &d) != cudaSuccess) return FFTC_ERR_ALLOC;
            const float2 *d_lo = (const float2 *)d;
            if (plan_upload(p, hi.data(), hi.size() * sizeof(float2), &d) != cudaSuccess) return FFTC_ERR_ALLOC;
            const float2 *d_hi = (const float2 *)d;
            // the whole inter-pass diagonal of this length in pass-1 layout (entry t' K + b =
            // w_n^(b t'), one rounding), shared by every row of the class
            std::vector<float2> full((size_t)nn);
            for (int64_t tp = 0; tp < M; ++tp)
                for (int64_t bb = 0; bb < K; ++bb) {
                    double cc, ss;
                    unit_root(tp * bb, nn, &cc, &ss);
                    full[(size_t)(tp * K + bb)] = make_float2((float)cc, (float)-ss);
                }
            if (plan_upload(p, full.data(), full.size() * sizeof(float2), &d) != cudaSuccess) return FFTC_ERR_ALLOC;
            const float2 *d_full = (const float2 *)d;
            for (int64_t id : ids) {
                const int conj = dir[id] == 1 ? 1 : 0;
                PassParams a{};
                a.in_user = 1;
                a.in = reinterpret_cast<const float *>((intptr_t)(off[id] * 8));
                a.out = reinterpret_cast<float *>(ws + ws_off);
                a.total_lines = K;
                a.log_lpt = logk;
                a.in_tr = a.out_tr = nn;
                a.in_line = a.out_line = 1;
                a.in_elem = a.out_elem = K;
                a.tw = tw1;
                a.tw2_lo = d_lo;
                a.tw2_hi = d_hi;
                a.tw2_full = d_full;
                a.log_n2 = logn;
                a.tw2_lo_bits = lob;
                a.conj_in = conj;
                PassParams b{};
                b.in = reinterpret_cast<const float *>(ws + ws_off);
                b.out_user = 1;
                b.out = reinterpret_cast<float *>((intptr_t)(off[id] * 8));
                b.total_lines = M;
                b.log_lpt = logm;
                b.in_tr = b.out_tr = nn;
                b.in_line = K;
                b.in_elem = 1;
                b.out_line = 1;
                b.out_elem = M;
                b.tw = tw2;
                b.conj_out = conj;
                const int pa = (int)u->params.size();
                u->params.push_back(a);
                const int pb = (int)u->params.size();
                u->params.push_back(b);
                const int done = n_done++;
                const int64_t t1 = K / kBranches[b1].lines, t2 = M / kBranches[b2].lines;
                for (int64_t t = 0; t < t1; ++t) p1.push_back(WorkItem{b1, pa, (int32_t)t, -1, 0, done});
                queued_bytes += 8.0 * nn;
                Pending pd;
                pd.release = queued_bytes + lag_bytes;
                for (int64_t t = 0; t < t2; ++t) pd.items.push_back(WorkItem{b2, pb, (int32_t)t, done, (int32_t)t1, -1});
                pend.push_back(pd);
                while (pend_head < pend.size() && pend[pend_head].release <= queued_bytes) {
                    p1.insert(p1.end(), pend[pend_head].items.begin(), pend[pend_head].items.end());
                    ++pend_head;
                }
                ws_off += nn;
            }
        }
    }
    for (; pend_head < pend.size(); ++pend_head) p2.insert(p2.end(), pend[pend_head].items.begin(), pend[pend_head].items.end());
    if (env_int("FFTC_TEST_UNREACHABLE_WAIT", 0)) {  // test hook: a dependency nothing satisfies
        for (WorkItem &w : p1)
            if (w.wait_idx >= 0) w.wait_target += 1;
        for (WorkItem &w : p2) w.wait_target += 1;
    }
    u->items = p1;
    u->items.insert(u->items.end(), p0.begin(), p0.end());
    u->items.insert(u->items.end(), p2.begin(), p2.end());
    u->n_ctrl = 1 + n_done;

    if (plan_upload(p, u->items.data(), u->items.size() * sizeof(WorkItem), &d) != cudaSuccess) return FFTC_ERR_ALLOC;
    u->d_items = (WorkItem *)d;
    if (plan_upload(p, u->params.data(), u->params.size() * sizeof(PassParams), &d) != cudaSuccess)
        return FFTC_ERR_ALLOC;
    u->d_params = (PassParams *)d;
    {
        std::vector<int8_t> bt(3 * kNumBranches);
        for (int i = 0; i < kNumBranches; ++i) {
            bt[i] = (int8_t)kBranches[i].logl;
            bt[kNumBranches + i] = (int8_t)std::min(kBranches[i].lines, 127);
            bt[2 * kNumBranches + i] = (int8_t)kBranches[i].kind;
        }
        if (plan_upload(p, bt.data(), bt.size(), &d) != cudaSuccess) return FFTC_ERR_ALLOC;
        u->d_branch = (int8_t *)d;
    }
    if (plan_alloc(p, (size_t)u->n_ctrl * sizeof(unsigned int), &d) != cudaSuccess) return FFTC_ERR_ALLOC;
    u->d_ctrl = (unsigned int *)d;
    if (plan_alloc(p, 16, &d) != cudaSuccess) return FFTC_ERR_ALLOC;
    p->d_err = (int *)d;
    if (cudaMemset(p->d_err, 0, 16) != cudaSuccess) return FFTC_ERR_CUDA;

    // launch shape: every SM full of resident CTAs
    int smem = 0;
    for (int i = 0; i < kNumBranches; ++i) smem = std::max(smem, kBranches[i].smem);
    u->smem = smem;
    u->kfunc = (void *)k_uneven<kUnevenCtasPerSm>;
    if (cudaFuncSetAttribute(u->kfunc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return FFTC_ERR_CUDA;
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, u->kfunc, kUnevenThreads, smem) != cudaSuccess)
        return FFTC_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) return FFTC_ERR_CUDA;
    u->grid = std::max(1, per_sm) * sms;
    u->args.spin_limit = (long long)env_int("FFTC_SPIN_LIMIT", 20000000);
    u->args.pf_ahead = env_int("FFTC_UNEVEN_PF", 0) ? u->grid : 0;  // measured slower: off by default
    if (build_graph(u, p->d_err, nullptr) != cudaSuccess) return FFTC_ERR_CUDA;
    return FFTC_OK;
}


// ---------------------------------------------------------------------------
// autotuner: per length class, time each candidate factorisation inside the
// persistent kernel and keep the fastest (cached per device; FFTC_TUNE_CACHE names
// an optional file that carries the choices across processes)
// ---------------------------------------------------------------------------
static std::mutex g_tune_mu;
static std::map<std::pair<std::string, int>, int> g_tuned;  // (device name, log n) -> class code
static bool g_tune_file_read = false;

// every compiled configuration of a length class: the split (single pass or n = M K) and the
// elements per thread (which fix the tile shape and the stages per pass)
static std::vector<int> candidates(int logn) {
    std::vector<int> c;
    for (int logm = 0; logm <= 8; ++logm) {
        if (logm > 0 && logm < 6) continue;
        if (logm > 0 && (logn - logm < 6 || logn - logm > 8)) continue;
        for (int ev = 0; ev <= 2; ++ev) {
            ClassCfg cc;
            cc.logm = logm;
            cc.ev = ev;
            if (ev == 2 && logm > 0 && cols_branch(logm, logn - logm, 2) == cols_branch(logm, logn - logm, 0) &&
                rowst_branch(logn - logm, logm, 2) == rowst_branch(logn - logm, logm, 0))
                continue;  // the same branches as the default variant
            if (class_supported(logn, cc)) c.push_back(cc.code());
        }
    }
    return c;
}

static int fixed_choice(int logn, void *ctx) {
    (void)logn;
    return *static_cast<int *>(ctx);
}

// Time one candidate: `rows` contiguous rows of length 2^logn, forward, 64 MiB in.
static double time_candidate(int device, int logn, int code, void *d_in, void *d_out, int64_t rows) {
    fftc_plan_s tp;
    tp.magic = FFTC_PLAN_MAGIC;
    tp.device = device;
    std::vector<int64_t> n((size_t)rows, int64_t(1) << logn), off((size_t)rows);
    std::vector<int8_t> dir((size_t)rows, -1);
    for (int64_t i = 0; i < rows; ++i) off[(size_t)i] = i << logn;
    int choice = code;
    double best = -1.0;
    if (build_state(&tp, rows, n.data(), dir.data(), off.data(), fixed_choice, &choice) == FFTC_OK) {
        cudaStream_t st;
        cudaEvent_t e0, e1;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess) {
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            bool ok = uneven_run(&tp, d_in, d_out, st) == FFTC_OK;  // warm-up
            for (int rep = 0; ok && rep < 3; ++rep) {
                cudaEventRecord(e0, st);
                ok = uneven_run(&tp, d_in, d_out, st) == FFTC_OK;
                cudaEventRecord(e1, st);
                float ms = 0.f;
                if (ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
                    best = (best < 0 || ms < best) ? ms : best;
                else
                    ok = false;
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            cudaStreamDestroy(st);
        }
    }
    uneven_free(&tp);
    plan_free_device(&tp);
    return best;
}

static void read_tune_file(const std::string &dev) {
    const char *path = getenv("FFTC_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char line[512], name[256];
    int logn, logm, ev;
    while (fgets(line, sizeof(line), f))  // the file also holds other planners' lines
        if (sscanf(line, "uneven %255[^|]|%d %d %d", name, &logn, &logm, &ev) == 4 && dev == name) {
            ClassCfg c;
            c.logm = logm;
            c.ev = ev;
            g_tuned[std::make_pair(dev, logn)] = c.code();
        }
    fclose(f);
}

// one line per choice: "uneven <device name>|<log2 n> <log2 M (0: one pass)> <tile variant>"
// (0: the default elements per thread, 1: half of them, 2: 16 on every line length)
static void append_tune_file(const std::string &dev, int logn, int code) {
    const char *path = getenv("FFTC_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    const ClassCfg c = ClassCfg::decode(code);
    fprintf(f, "uneven %s|%d %d %d\n", dev.c_str(), logn, c.logm, c.ev);
    fclose(f);
}

struct TuneCtx {
    int device;
    std::string dev_name;
    void *d_in, *d_out;
    int64_t elems;
};

static int tuned_choice(int logn, void *vctx) {
    TuneCtx *ctx = static_cast<TuneCtx *>(vctx);
    char name[64];
    snprintf(name, sizeof(name), "FFTC_UNEVEN_LOGM_%d", logn);
    const int forced = env_int(name, -1);
    snprintf(name, sizeof(name), "FFTC_UNEVEN_EV_%d", logn);
    const int forced_ev = env_int(name, 0);
    if (forced >= 0) return forced | (forced_ev << 8);
    std::vector<int> cand = candidates(logn);
    if (cand.empty()) return -1;
    const int dflt = logn <= 12 ? 0 : logn / 2;
    if (cand.size() == 1 || env_int("FFTC_TUNE", 1) == 0) return dflt;
    auto key = std::make_pair(ctx->dev_name, logn);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) return it->second;
    if (!ctx->d_in) {  // tuning buffers, freed when the plan is built
        if (cudaMalloc(&ctx->d_in, (size_t)ctx->elems * 8) != cudaSuccess) ctx->d_in = nullptr;
        if (ctx->d_in && cudaMalloc(&ctx->d_out, (size_t)ctx->elems * 8) != cudaSuccess) ctx->d_out = nullptr;
        if (!ctx->d_in || !ctx->d_out) return dflt;
        cudaMemset(ctx->d_in, 0, (size_t)ctx->elems * 8);
    }
    const int64_t rows = ctx->elems >> logn;
    int best = dflt;
    double best_ms = -1.0;
    for (int c : cand) {
        const double ms = time_candidate(ctx->device, logn, c, ctx->d_in, ctx->d_out, rows);
        if (ms > 0 && (best_ms < 0 || ms < best_ms)) {
            best_ms = ms;
            best = c;
        }
    }
    g_tuned[key] = best;
    append_tune_file(ctx->dev_name, logn, best);
    return best;
}

fftc_status uneven_build(fftc_plan_s *p, int64_t count, const int64_t *n, const int8_t *dir, const int64_t *off) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    TuneCtx ctx{};
    ctx.device = p->device;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, p->device) != cudaSuccess) return FFTC_ERR_CUDA;
    ctx.dev_name = prop.name;
    ctx.elems = int64_t(1) << 23;  // 64 MiB per tuning buffer
    if (!g_tune_file_read) {
        read_tune_file(ctx.dev_name);
        g_tune_file_read = true;
    }
    fftc_status s = build_state(p, count, n, dir, off, tuned_choice, &ctx);
    if (ctx.d_in) cudaFree(ctx.d_in);
    if (ctx.d_out) cudaFree(ctx.d_out);
    return s;
}


}  // namespace fftc

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

#include "fftc_fourstep_l2.cuh"
#include "fftc_plan.h"

namespace fftc {

extern const FsEntry kFsIlTable[], kFsSplitTable[];
extern const int kFsIlCount, kFsSplitCount;



static const FsEntry *find_fs(int logn, int lay) {
    const FsEntry *t = lay == LAYOUT_IL ? kFsIlTable : kFsSplitTable;
    const int n = lay == LAYOUT_IL ? kFsIlCount : kFsSplitCount;
    for (int i = 0; i < n; ++i)
        if (t[i].logn == logn) return &t[i];
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
    // test hook: every wait is for a count nothing reaches, so each one runs out
    a.wait_bias = env_int_fs("FFTC_TEST_UNREACHABLE_WAIT", 0) ? (1u << 30) : 0u;
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

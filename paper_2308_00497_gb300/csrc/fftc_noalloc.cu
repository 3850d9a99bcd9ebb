// fftc_execute_noalloc: the two-pass (four-step) transform without any device
// allocation, for callers that are not allowed to allocate device memory.
//
// The inter-pass workspace and the twiddle tables live in file-scope __device__
// arrays of fixed size, which every GPU that loads libfftc.so holds until the
// process exits. Host code must not pass those arrays' names to a kernel (in host
// code they are host-side stand-ins); the device addresses are looked up with
// cudaGetSymbolAddress, with the device current. The first call on a device does the
// set-up (addresses, kernel choice per size, one synchronous upload of the tables);
// every later call looks the scratch address up again and redoes the set-up if it has
// changed (a device reset or a new primary context reloads the module, whose arrays are
// then new and zero-filled).
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "../../include/fftc.h"
#include "fftc_plan.h"

namespace fftc {
namespace {

constexpr int kMinLog = 14, kMaxLog = 20;     // the sizes that need a workspace
constexpr int kNumLogs = kMaxLog - kMinLog + 1;
constexpr int64_t kScratchElems = int64_t(1) << 21;  // n * batch limit: 16 MiB of complex64
constexpr int kTabPerLog = 4096;              // stage tables of both passes + two inter-pass tables
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float2 g_noalloc_scratch[kScratchElems];
static __device__ __align__(256) float2 g_noalloc_tables[kNumLogs * kTabPerLog];

struct SizeSetup {
    bool ok = false;  // kernels found and prepared for both layouts
    int logm, e1, e2, lo_bits, pf;
    const KernelEntry *k1[2], *k2[2];  // per layout: pass 1 (COLS), pass 2 (ROWST)
    int off_tw1, off_tw2, off_lo, off_hi;  // table offsets (float2 entries) inside this size's block
};

struct DeviceSetup {
    bool ready = false;
    float2 *scratch = nullptr;  // device address of g_noalloc_scratch
    float2 *tables = nullptr;   // device address of g_noalloc_tables
    SizeSetup size[kNumLogs];
};

std::mutex g_mu;
DeviceSetup g_dev[kMaxDevices];

fftc_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return FFTC_OK;
    return e == cudaErrorMemoryAllocation ? FFTC_ERR_ALLOC : FFTC_ERR_CUDA;
}

// the compiled kernel for a four-step pass: the compile-time stride variant if there is
// one, else the runtime-stride kernel of the same shape
const KernelEntry *pass_kernel(int kind, int logl, int loge, int lines, int lin, int lout, int logx) {
    const KernelEntry *k = find_kernel(kind, logl, loge, lines, lin, lout, 0, logx);
    return k ? k : find_kernel(kind, logl, loge, lines, lin, lout, 0, 0);
}

// Kernels and tables of one size; a size whose kernels are missing stays unsupported
// without affecting the others.
void setup_size(int logn, SizeSetup &s, float2 *blk) {
    s.ok = false;
    const FourStepChoice fc = choose_four_step(logn, LAYOUT_IL);  // plain kernels of the same shapes
    s.logm = fc.logm;
    s.e1 = fc.e1;
    s.e2 = fc.e2;
    s.pf = fc.pf;
    const int logk = logn - s.logm;
    for (int lay = 0; lay < 2; ++lay) {
        s.k1[lay] = pass_kernel(KIND_COLS, s.logm, s.e1, fc.c1, lay, LAYOUT_IL, logk);
        s.k2[lay] = pass_kernel(KIND_ROWST, logk, s.e2, fc.c2, LAYOUT_IL, lay, s.logm);
        if (!s.k1[lay] || !s.k2[lay]) return;
        if (s.k1[lay]->prepare() != cudaSuccess || s.k2[lay]->prepare() != cudaSuccess) return;
    }
    std::vector<float2> t1, t2;
    stage_twiddles(s.logm, s.e1, t1);
    stage_twiddles(logk, s.e2, t2);
    s.lo_bits = (logn + 1) / 2;
    const int64_t n = int64_t(1) << logn, nlo = int64_t(1) << s.lo_bits, nhi = n >> s.lo_bits;
    s.off_tw1 = 0;
    s.off_tw2 = s.off_tw1 + (int)t1.size();
    s.off_lo = s.off_tw2 + (int)t2.size();
    s.off_hi = s.off_lo + (int)nlo;
    if (s.off_hi + nhi > kTabPerLog) return;
    for (size_t i = 0; i < t1.size(); ++i) blk[s.off_tw1 + i] = t1[i];
    for (size_t i = 0; i < t2.size(); ++i) blk[s.off_tw2 + i] = t2[i];
    for (int64_t m = 0; m < nlo; ++m) {
        double c, sn;
        unit_root(m, n, &c, &sn);
        blk[s.off_lo + m] = make_float2((float)c, (float)-sn);
    }
    for (int64_t m = 0; m < nhi; ++m) {
        double c, sn;
        unit_root(m * nlo, n, &c, &sn);
        blk[s.off_hi + m] = make_float2((float)c, (float)-sn);
    }
    s.ok = true;
}

// Look the arrays up on the current device; set the device up when it has not been, or
// when the scratch address changed since (the module was reloaded). A failed set-up is
// not cached, so a later call retries it.
fftc_status ensure_device(DeviceSetup &d) {
    void *p = nullptr;
    fftc_status st = cuda_status(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    if (st != FFTC_OK) return st;
    if (!p) return FFTC_ERR_CUDA;
    if (d.ready && p == (void *)d.scratch) return FFTC_OK;
    d.ready = false;
    d.scratch = (float2 *)p;
    p = nullptr;
    if ((st = cuda_status(cudaGetSymbolAddress(&p, g_noalloc_tables))) != FFTC_OK) return st;
    if (!p) return FFTC_ERR_CUDA;
    d.tables = (float2 *)p;
    std::vector<float2> host((size_t)kNumLogs * kTabPerLog, make_float2(0.f, 0.f));
    for (int logn = kMinLog; logn <= kMaxLog; ++logn)
        setup_size(logn, d.size[logn - kMinLog], host.data() + (size_t)(logn - kMinLog) * kTabPerLog);
    if ((st = cuda_status(cudaMemcpy(d.tables, host.data(), host.size() * sizeof(float2), cudaMemcpyHostToDevice))) !=
        FFTC_OK)
        return st;
    d.ready = true;
    return FFTC_OK;
}

}  // namespace
}  // namespace fftc

using namespace fftc;

extern "C" fftc_status fftc_execute_noalloc(int64_t n, int64_t batch, fftc_layout layout, fftc_direction direction,
                                            const void *in, void *out, void *stream) {
    if (layout != FFTC_LAYOUT_INTERLEAVED && layout != FFTC_LAYOUT_SPLIT) return FFTC_ERR_INVALID_VALUE;
    if (direction != FFTC_FORWARD && direction != FFTC_INVERSE) return FFTC_ERR_INVALID_VALUE;
    if (batch < 0) return FFTC_ERR_INVALID_VALUE;
    if (n < (int64_t(1) << kMinLog) || n > (int64_t(1) << kMaxLog) || (n & (n - 1)) != 0)
        return FFTC_ERR_UNSUPPORTED_SIZE;
    if (batch > kScratchElems / n) return FFTC_ERR_UNSUPPORTED_SIZE;
    if (batch == 0) return FFTC_OK;
    if (!in || !out) return FFTC_ERR_INVALID_VALUE;
    if ((reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(out) & 15)) return FFTC_ERR_MISALIGNED;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FFTC_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return FFTC_ERR_INVALID_VALUE;
    DeviceSetup *d = &g_dev[dev];
    {
        std::lock_guard<std::mutex> lk(g_mu);
        fftc_status s = ensure_device(*d);
        if (s != FFTC_OK) return s;
    }
    int logn = 0;
    while ((int64_t(1) << logn) < n) ++logn;
    const SizeSetup &s = d->size[logn - kMinLog];
    if (!s.ok) return FFTC_ERR_UNSUPPORTED_SIZE;
    const int lay = layout == FFTC_LAYOUT_SPLIT ? LAYOUT_SPLIT : LAYOUT_IL;
    const int logk = logn - s.logm;
    const int64_t M = int64_t(1) << s.logm, K = int64_t(1) << logk;
    const int64_t plane = lay == LAYOUT_SPLIT ? n * batch : 0;
    const float2 *tab = d->tables + (size_t)(logn - kMinLog) * kTabPerLog;
    const int inv = direction == FFTC_INVERSE ? 1 : 0;
    cudaStream_t st = (cudaStream_t)stream;

    PassParams a{};
    a.in = (const float *)in;
    a.out = (float *)d->scratch;
    a.in_plane = plane;
    a.total_lines = batch * K;
    a.log_lpt = logk;
    a.in_tr = n;
    a.in_line = 1;
    a.in_elem = K;
    a.out_tr = n;
    a.out_line = 1;
    a.out_elem = K;
    a.tw = tab + s.off_tw1;
    a.tw2_lo = tab + s.off_lo;
    a.tw2_hi = tab + s.off_hi;
    a.log_n2 = logn;
    a.tw2_lo_bits = s.lo_bits;
    a.conj_in = inv;
    a.pf_tiles = s.pf ? -1 : 0;
    if (s.k1[lay]->launch(a, st) != cudaSuccess) return FFTC_ERR_CUDA;

    PassParams b{};
    b.in = (const float *)d->scratch;
    b.out = (float *)out;
    b.out_plane = plane;
    b.total_lines = batch * M;
    b.log_lpt = s.logm;
    b.in_tr = n;
    b.in_line = K;
    b.in_elem = 1;
    b.out_tr = n;
    b.out_line = 1;
    b.out_elem = M;
    b.tw = tab + s.off_tw2;
    b.post_line_mul = 1;
    b.post_elem_mul = M;
    b.conj_out = inv;
    if (s.k2[lay]->launch(b, st) != cudaSuccess) return FFTC_ERR_CUDA;
    return FFTC_OK;
}

// C ABI of libfftc.so: plan creation (radix/pass planning, FP64 twiddle tables,
// workspace), execution and error reporting. See include/fftc.h.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <set>
#include <vector>

#include "../../include/fftc.h"
#include "fftc_internal.h"
#include "fftc_plan.h"

using namespace fftc;

namespace fftc {

// ---------------------------------------------------------------------------
// schedule mirror and registry
// ---------------------------------------------------------------------------
HostSched host_sched(int logl, int loge) {
    HostSched h{};
    if (loge > logl) loge = logl;
    h.S = (logl + loge - 1) / loge;
    const int rem = logl % loge;
    int acc = 0;
    for (int s = 0; s < h.S; ++s) {
        h.lr[s] = (rem && s == h.S - 1) ? rem : loge;
        h.lns[s] = acc;
        acc += h.lr[s];
    }
    int o = 0;
    for (int s = 1; s < h.S; ++s) o += ((1 << h.lr[s]) - 1) << h.lns[s];
    h.tw_total = o;
    return h;
}

const KernelEntry *find_kernel(int kind, int logl, int loge, int lines, int lin, int lout, int prec, int logx,
                               int pipe) {
    for (int i = 0; i < kernel_count(); ++i) {
        const KernelEntry *e = kernel_at(i);
        if (e->kind == kind && e->logl == logl && e->loge == loge && e->lines == lines && e->lin == lin &&
            e->lout == lout && e->prec == prec && e->logx == logx && e->pipe == pipe)
            return e;
    }
    return nullptr;
}

const KernelEntry *find_pipe_rows(int logl, int lay) {
    for (int i = 0; i < kernel_count(); ++i) {
        const KernelEntry *e = kernel_at(i);
        if (e->pipe > 0 && e->prec == 0 && e->kind == KIND_ROWS && e->logl == logl && e->lin == lay) return e;
    }
    return nullptr;
}

// cos and sin of 2*pi*m/L in FP64 with exact integer reduction of the angle to
// the first octant (the fraction m/L is kept as an exact ratio of integers).
void unit_root(int64_t m, int64_t L, double *cosv, double *sinv) {
    m %= L;
    if (m < 0) m += L;
    int64_t num = m, den = L;
    double sc = 1.0, ss = 1.0;
    bool swap = false;
    if (2 * num >= den) {  // f >= 1/2: f - 1/2, both parts negate
        num = 2 * num - den;
        den *= 2;
        sc = -sc;
        ss = -ss;
    }
    if (4 * num > den) {  // f > 1/4: 1/2 - f, cosine negates
        num = den - 2 * num;
        den *= 2;
        sc = -sc;
    }
    if (8 * num > den) {  // f > 1/8: 1/4 - f, cosine and sine swap
        num = den - 4 * num;
        den *= 4;
        swap = true;
    }
    const double th = 6.283185307179586476925286766559 * ((double)num / (double)den);
    double c = std::cos(th), s = std::sin(th);
    if (swap) {
        double t = c;
        c = s;
        s = t;
    }
    *cosv = sc * c;
    *sinv = ss * s;
}

// w_L^e = exp(-2 pi i e / L), rounded once to float.
static float2 omega_f32(int64_t e, int64_t L) {
    double c, s;
    unit_root(e, L, &c, &s);
    return make_float2((float)c, (float)-s);
}

void stage_twiddles(int logl, int loge, std::vector<float2> &out) {
    HostSched h = host_sched(logl, loge);
    out.assign(h.tw_total > 0 ? h.tw_total : 1, make_float2(1.f, 0.f));
    int off = 0;
    for (int s = 1; s < h.S; ++s) {
        const int R = 1 << h.lr[s], Ns = 1 << h.lns[s];
        for (int t = 1; t < R; ++t)
            for (int k = 0; k < Ns; ++k) out[off + (t - 1) * Ns + k] = omega_f32((int64_t)t * k, (int64_t)Ns * R);
        off += (R - 1) * Ns;
    }
}

}  // namespace fftc

// ---------------------------------------------------------------------------
// error state and plan registry
// ---------------------------------------------------------------------------
static thread_local fftc_status g_last_error = FFTC_OK;
static std::mutex g_mu;
static std::set<fftc_plan_s *> *g_live = nullptr;  // intentionally leaked: safe at exit

static void register_plan(fftc_plan_s *p) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_live) g_live = new std::set<fftc_plan_s *>();
    g_live->insert(p);
}
static bool is_live(const fftc_plan_s *p) {
    std::lock_guard<std::mutex> lk(g_mu);
    return p && g_live && g_live->count(const_cast<fftc_plan_s *>(p)) && p->magic == FFTC_PLAN_MAGIC;
}
static bool unregister_plan(fftc_plan_s *p) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_live || !g_live->count(p)) return false;
    g_live->erase(p);
    return true;
}

static fftc_plan fail(fftc_status s, fftc_plan_s *p = nullptr) {
    g_last_error = s;
    if (p) {
        plan_destroy_extra(p);
        plan_free_device(p);
        delete p;
    }
    return nullptr;
}

static bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
static int log2i(int64_t v) {
    int r = 0;
    while ((int64_t(1) << r) < v) ++r;
    return r;
}

namespace fftc {

void plan_free_device(fftc_plan_s *p) {
    for (void *ptr : p->dev_allocs) cudaFree(ptr);
    p->dev_allocs.clear();
}

cudaError_t plan_alloc(fftc_plan_s *p, size_t bytes, void **out) {
    *out = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(out, bytes);
    if (e == cudaSuccess) p->dev_allocs.push_back(*out);
    return e;
}

void plan_release(fftc_plan_s *p, void *ptr) {
    for (size_t i = 0; i < p->dev_allocs.size(); ++i)
        if (p->dev_allocs[i] == ptr) {
            cudaFree(ptr);
            p->dev_allocs.erase(p->dev_allocs.begin() + (long)i);
            return;
        }
}

cudaError_t plan_upload(fftc_plan_s *p, const void *host, size_t bytes, void **out) {
    cudaError_t e = plan_alloc(p, bytes, out);
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*out, host, bytes, cudaMemcpyHostToDevice);
}

}  // namespace fftc

extern "C" {

fftc_status fftc_get_last_error(void) { return g_last_error; }

const char *fftc_status_string(fftc_status s) {
    switch (s) {
        case FFTC_OK: return "FFTC_OK";
        case FFTC_ERR_INVALID_VALUE: return "FFTC_ERR_INVALID_VALUE";
        case FFTC_ERR_UNSUPPORTED_SIZE: return "FFTC_ERR_UNSUPPORTED_SIZE";
        case FFTC_ERR_MISALIGNED: return "FFTC_ERR_MISALIGNED";
        case FFTC_ERR_ALLOC: return "FFTC_ERR_ALLOC";
        case FFTC_ERR_CUDA: return "FFTC_ERR_CUDA";
        case FFTC_ERR_INVALID_PLAN: return "FFTC_ERR_INVALID_PLAN";
        case FFTC_ERR_TIMEOUT: return "FFTC_ERR_TIMEOUT";
    }
    return "FFTC_ERR_UNKNOWN";
}

fftc_plan fftc_plan_create(int64_t n, int64_t batch, fftc_layout layout, fftc_direction direction,
                           fftc_precision precision) {
    if (layout != FFTC_LAYOUT_INTERLEAVED && layout != FFTC_LAYOUT_SPLIT) return fail(FFTC_ERR_INVALID_VALUE);
    if (direction != FFTC_FORWARD && direction != FFTC_INVERSE) return fail(FFTC_ERR_INVALID_VALUE);
    if ((int)precision < (int)FFTC_FP32 || (int)precision > (int)FFTC_FP64) return fail(FFTC_ERR_INVALID_VALUE);
    if (batch < 0) return fail(FFTC_ERR_INVALID_VALUE);
    if (n < 2 || n > (int64_t(1) << 24)) return fail(FFTC_ERR_UNSUPPORTED_SIZE);
    const bool tc = precision != FFTC_FP32 && precision != FFTC_FP64;
    if (!is_pow2(n) && (!mixed_supported(n) || tc)) return fail(FFTC_ERR_UNSUPPORTED_SIZE);
    // FP64 and non-power-of-two lengths run the runtime-radix path: it needs n = M K with
    // both factors at most one CTA's line
    if ((!is_pow2(n) || precision == FFTC_FP64) && mixed_split(n, precision == FFTC_FP64) == 0)
        return fail(FFTC_ERR_UNSUPPORTED_SIZE);
    if (batch > (int64_t(1) << 40) / n) return fail(FFTC_ERR_UNSUPPORTED_SIZE);

    fftc_plan_s *p = new (std::nothrow) fftc_plan_s();
    if (!p) return fail(FFTC_ERR_ALLOC);
    p->magic = FFTC_PLAN_MAGIC;
    p->n = n;
    p->logn = log2i(n);
    p->batch = batch;
    p->layout = layout;
    p->direction = direction;
    p->precision = precision;
    if (cudaGetDevice(&p->device) != cudaSuccess) return fail(FFTC_ERR_CUDA, p);

    fftc_status st = plan_build(p);
    if (st != FFTC_OK) return fail(st, p);
    register_plan(p);
    g_last_error = FFTC_OK;
    return p;
}

fftc_status fftc_destroy(fftc_plan plan) {
    if (!plan) return FFTC_OK;
    if (!unregister_plan(plan)) return FFTC_ERR_INVALID_PLAN;
    plan_destroy_extra(plan);
    plan_probe_free(plan);
    plan_free_device(plan);
    plan->magic = 0;
    delete plan;
    return FFTC_OK;
}

int64_t fftc_plan_bytes(fftc_plan plan) {
    if (!is_live(plan)) return 0;
    return plan->total_elems * (plan->precision == FFTC_FP64 ? 16 : 8);
}

fftc_status fftc_plan_info(fftc_plan plan, int *passes, int *radices, int *n_radices) {
    if (!is_live(plan)) return FFTC_ERR_INVALID_PLAN;
    int cnt = 0;
    int tmp[32];
    if (plan->uneven) {
        if (passes) *passes = 1;
        HostSched h = host_sched(uneven_max_logn(plan), 4);
        for (int s = 0; s < h.S && cnt < 32; ++s) tmp[cnt++] = 1 << h.lr[s];
    } else if (passes) {
        *passes = plan->npasses;
    }
    if (plan->mixed) cnt = mixed_radix_list(plan, tmp, 32);
    if (plan->nd) cnt = 0;  // several 1D factorisations: the pass count alone is reported
    const int nsched = (plan->fs || plan->cluster) ? 2 : plan->npasses;
    for (int i = 0; i < nsched && !plan->uneven && !plan->mixed && !plan->nd; ++i) {
        const PassPlan &pp = plan->pass[i];
        HostSched h = host_sched(pp.logl, pp.loge);
        for (int s = 0; s < h.S && cnt < 32; ++s) tmp[cnt++] = 1 << h.lr[s];
    }
    if (radices)
        for (int i = 0; i < cnt && i < 16; ++i) radices[i] = tmp[i];
    if (n_radices) *n_radices = cnt;
    return FFTC_OK;
}

fftc_status fftc_plan_split(fftc_plan plan, int64_t *m, int64_t *k) {
    if (!is_live(plan)) return FFTC_ERR_INVALID_PLAN;
    if (plan->uneven || plan->nd) return FFTC_ERR_INVALID_VALUE;
    int64_t mm = plan->n, kk = 1;
    if (plan->mixed) {
        mm = mixed_plan_split(plan);
        kk = plan->n / mm;
    } else if (plan->npasses >= 2 || plan->fs || plan->cluster) {
        mm = int64_t(1) << plan->pass[0].logl;
        kk = plan->n / mm;
    }
    if (m) *m = mm;
    if (k) *k = kk;
    return FFTC_OK;
}

fftc_status fftc_execute(fftc_plan plan, const void *in, void *out, void *stream) {
    if (!is_live(plan)) return FFTC_ERR_INVALID_PLAN;
    if (plan->total_elems == 0) return FFTC_OK;
    if (!in || !out) return FFTC_ERR_INVALID_VALUE;
    if ((reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(out) & 15))
        return FFTC_ERR_MISALIGNED;
    return plan_run(plan, in, out, nullptr, 0.f, (cudaStream_t)stream);
}

fftc_status fftc_plan_tune(fftc_plan plan, int reps) {
    if (!is_live(plan)) return FFTC_ERR_INVALID_PLAN;
    if (reps < 1 || reps > 1000) return FFTC_ERR_INVALID_VALUE;
    return plan_tune(plan, reps);
}

fftc_plan fftc_plan_create_nd(int rank, const int64_t *dims, int64_t batch, fftc_layout layout,
                              fftc_direction direction, fftc_precision precision) {
    if (rank < 2 || rank > 3 || !dims || batch < 0) return fail(FFTC_ERR_INVALID_VALUE);
    if (layout != FFTC_LAYOUT_INTERLEAVED && layout != FFTC_LAYOUT_SPLIT) return fail(FFTC_ERR_INVALID_VALUE);
    if (direction != FFTC_FORWARD && direction != FFTC_INVERSE) return fail(FFTC_ERR_INVALID_VALUE);
    if ((int)precision < (int)FFTC_FP32 || (int)precision > (int)FFTC_FP64) return fail(FFTC_ERR_INVALID_VALUE);
    if (precision != FFTC_FP32 && precision != FFTC_FP64) return fail(FFTC_ERR_UNSUPPORTED_SIZE);
    int64_t per = 1;
    for (int a = 0; a < rank; ++a) {
        const int64_t d = dims[a];
        const bool ok = a == rank - 1 ? (d >= 2 && d <= (int64_t(1) << 24) && (is_pow2(d) || mixed_supported(d)))
                                      : nd_axis_supported(d, precision == FFTC_FP64);
        if (!ok) return fail(FFTC_ERR_UNSUPPORTED_SIZE);
        per *= d;
        if (per > (int64_t(1) << 30)) return fail(FFTC_ERR_UNSUPPORTED_SIZE);
    }
    if (batch > (int64_t(1) << 30) / per) return fail(FFTC_ERR_UNSUPPORTED_SIZE);
    fftc_plan_s *p = new (std::nothrow) fftc_plan_s();
    if (!p) return fail(FFTC_ERR_ALLOC);
    p->magic = FFTC_PLAN_MAGIC;
    p->n = per;
    p->batch = batch;
    p->layout = layout;
    p->direction = direction;
    p->precision = precision;
    if (cudaGetDevice(&p->device) != cudaSuccess) return fail(FFTC_ERR_CUDA, p);
    fftc_status st = nd_build(p, rank, dims);
    if (st != FFTC_OK) return fail(st, p);
    register_plan(p);
    g_last_error = FFTC_OK;
    return p;
}

fftc_plan fftc_plan_create_uneven(int64_t count, const int64_t *n, const int8_t *direction, const int64_t *offset,
                                  fftc_layout layout, fftc_precision precision) {
    if (count < 1 || count > (int64_t(1) << 24) || !n || !direction || !offset) return fail(FFTC_ERR_INVALID_VALUE);
    if (layout != FFTC_LAYOUT_INTERLEAVED) return fail(FFTC_ERR_INVALID_VALUE);
    if (precision != FFTC_FP32) return fail(FFTC_ERR_INVALID_VALUE);
    for (int64_t i = 0; i < count; ++i)
        if (n[i] < 64 || n[i] > (int64_t(1) << 16) || !is_pow2(n[i])) return fail(FFTC_ERR_UNSUPPORTED_SIZE);
    fftc_plan_s *p = new (std::nothrow) fftc_plan_s();
    if (!p) return fail(FFTC_ERR_ALLOC);
    p->magic = FFTC_PLAN_MAGIC;
    p->layout = layout;
    p->precision = precision;
    p->batch = count;
    if (cudaGetDevice(&p->device) != cudaSuccess) return fail(FFTC_ERR_CUDA, p);
    fftc_status st = uneven_build(p, count, n, direction, offset);
    if (st != FFTC_OK) return fail(st, p);
    p->npasses = 1;
    register_plan(p);
    g_last_error = FFTC_OK;
    return p;
}

fftc_status fftc_execute_pointwise(fftc_plan plan, const void *in, void *out, const float *h, float scale,
                                   void *stream) {
    if (!is_live(plan)) return FFTC_ERR_INVALID_PLAN;
    if (plan->uneven || plan->precision != FFTC_FP32) return FFTC_ERR_INVALID_VALUE;
    if (plan->total_elems == 0) return FFTC_OK;
    if (!in || !out || !h) return FFTC_ERR_INVALID_VALUE;
    if ((reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(out) & 15) ||
        (reinterpret_cast<uintptr_t>(h) & 15))
        return FFTC_ERR_MISALIGNED;
    return plan_run(plan, in, out, h, scale, (cudaStream_t)stream);
}

fftc_status fftc_execute_host(fftc_plan plan, const void *host_in, void *host_out, void *dev_buf, void *stream) {
    if (!is_live(plan)) return FFTC_ERR_INVALID_PLAN;
    if (plan->total_elems == 0) return FFTC_OK;
    if (!host_in || !host_out || !dev_buf) return FFTC_ERR_INVALID_VALUE;
    if (reinterpret_cast<uintptr_t>(dev_buf) & 15) return FFTC_ERR_MISALIGNED;
    return host_execute(plan, host_in, host_out, dev_buf, (cudaStream_t)stream);
}

fftc_status fftc_stage_twiddles(int logl, int loge, float *out, int64_t capacity, int64_t *count) {
    if (loge < 1 || loge > logl || logl > 20 || !count) return FFTC_ERR_INVALID_VALUE;
    std::vector<float2> t;
    stage_twiddles(logl, loge, t);
    const int64_t used = host_sched(logl, loge).tw_total;
    *count = used;
    if (used > capacity || (used > 0 && !out)) return FFTC_ERR_INVALID_VALUE;
    for (int64_t i = 0; i < used; ++i) {
        out[2 * i] = t[(size_t)i].x;
        out[2 * i + 1] = t[(size_t)i].y;
    }
    return FFTC_OK;
}

fftc_status fftc_plan_timing(fftc_plan plan, int enable) {
    if (!is_live(plan)) return FFTC_ERR_INVALID_PLAN;
    plan_probe_free(plan);
    if (!enable) return FFTC_OK;
    const int slots = 4096;
    try {
        plan->probe_events.resize((size_t)3 * slots);
    } catch (...) {
        return FFTC_ERR_ALLOC;
    }
    for (size_t i = 0; i < plan->probe_events.size(); ++i) {
        if (cudaEventCreate(&plan->probe_events[i]) != cudaSuccess) {
            plan->probe_events.resize(i);
            plan_probe_free(plan);
            return FFTC_ERR_CUDA;
        }
    }
    plan->probe_slots = slots;
    plan->probe_used = 0;
    plan->probe_on = true;
    return FFTC_OK;
}

fftc_status fftc_plan_pass_times(fftc_plan plan, double *ms_per_pass, int *executes) {
    if (!is_live(plan)) return FFTC_ERR_INVALID_PLAN;
    double acc[2] = {0.0, 0.0};
    const int np = plan->npasses > 0 ? plan->npasses : 1;
    for (int s = 0; s < plan->probe_used; ++s) {
        cudaEvent_t *ev = &plan->probe_events[(size_t)3 * s];
        for (int i = 0; i < np && i < 2; ++i) {
            if (cudaEventSynchronize(ev[i + 1]) != cudaSuccess) return FFTC_ERR_CUDA;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) != cudaSuccess) return FFTC_ERR_CUDA;
            acc[i] += ms;
        }
    }
    if (ms_per_pass) {
        ms_per_pass[0] = acc[0];
        ms_per_pass[1] = acc[1];
    }
    if (executes) *executes = plan->probe_used;
    return FFTC_OK;
}

fftc_status fftc_plan_check(fftc_plan plan, void *stream) {
    if (!is_live(plan)) return FFTC_ERR_INVALID_PLAN;
    return plan_check_errors(plan, (cudaStream_t)stream);
}

}  // extern "C"

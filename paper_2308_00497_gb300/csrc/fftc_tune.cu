// Measurement-driven planning (FFTW's "measure" mode, the runtime search over
// decompositions that the paper leaves to future work, Section 6): candidate plans are
// timed on scratch buffers of the plan's size and the fastest is kept.
//   single pass: every registered rows kernel for (n, layout): plain, bulk-copy fed with
//                each landing-buffer count and refill point, each elements-per-thread
//                (the radix schedule of the line: radix 2^loge stages, remainder last)
//                and tile height;
//   four-step:   every split n = M K of Eq. 1 at the memory level with compiled kernels
//                for both passes, and for each split every column kernel for pass 1
//                (plain with and without the L2 prefetch, tensor-map fed; compile-time
//                or runtime stride; each radix schedule) and every transposed-row kernel
//                for pass 2, timed pass by pass; the split with the smallest sum wins.
// Tensor-core plans choose among the tensor-core kernels of their precision mode.
// Choices are cached per (n, batch, layout, direction, precision) for the process.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <map>
#include <string>
#include <mutex>
#include <tuple>
#include <vector>

#include "fftc_plan.h"

namespace fftc {

namespace {

struct Choice {
    int logm = 0;  // four-step split n = 2^logm * 2^(logn - logm) (unused for one pass)
    const KernelEntry *k1 = nullptr, *k2 = nullptr;
    int pf1 = 0;
    const ClusterEntry *cl = nullptr;  // the cluster single pass instead of the above
};

std::mutex g_tune_mu;
std::map<std::tuple<int64_t, int64_t, int, int, int>, Choice> g_tune_cache;
bool g_tune_file_read = false;

// FFTC_TUNE_CACHE, when set, names a text file that carries the choices across processes
// (FFTW's "wisdom"): one line per shape,
//   plan <device name>|<n> <batch> <layout> <direction> <precision> S <k1>
//   plan <device name>|<n> <batch> <layout> <direction> <precision> F <log2 M> <pf> <k1> <k2>
//   plan <device name>|<n> <batch> <layout> <direction> <precision> C <log2 n> <log2 n1> <loge> <R> <layout>
// with a kernel written as its registry identity "kind logl loge lines lin lout prec logx
// pipe". Lines whose kernels this build lacks are ignored (the shape is then timed again).
std::string device_name() {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "";
    return prop.name;
}

void put_kernel(std::string &out, const KernelEntry *k) {
    char b[160];
    snprintf(b, sizeof(b), " %d %d %d %d %d %d %d %d %d", k->kind, k->logl, k->loge, k->lines, k->lin, k->lout, k->prec,
             k->logx, k->pipe);
    out += b;
}

const KernelEntry *get_kernel(const char *&s) {
    int v[9], used = 0;
    if (sscanf(s, " %d %d %d %d %d %d %d %d %d%n", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5], &v[6], &v[7], &v[8],
               &used) != 9)
        return nullptr;
    s += used;
    return find_kernel(v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7], v[8]);
}

void read_tune_file() {
    const char *path = getenv("FFTC_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    const std::string dev = device_name();
    char line[512], name[256], kind;
    long long n, batch;
    int lay, dir, prec, used;
    while (fgets(line, sizeof(line), f)) {
        if (sscanf(line, "plan %255[^|]|%lld %lld %d %d %d %c%n", name, &n, &batch, &lay, &dir, &prec, &kind, &used) != 7 ||
            dev != name)
            continue;
        const char *rest = line + used;
        Choice c;
        bool ok = false;
        if (kind == 'S') {
            ok = (c.k1 = get_kernel(rest)) != nullptr;
        } else if (kind == 'F') {
            int u2 = 0;
            if (sscanf(rest, " %d %d%n", &c.logm, &c.pf1, &u2) == 2) {
                rest += u2;
                c.k1 = get_kernel(rest);
                c.k2 = c.k1 ? get_kernel(rest) : nullptr;
                ok = c.k1 && c.k2;
            }
        } else if (kind == 'C') {
            int v[5];
            if (sscanf(rest, " %d %d %d %d %d", &v[0], &v[1], &v[2], &v[3], &v[4]) == 5)
                for (int i = 0; i < cluster_kernel_count() && !ok; ++i) {
                    const ClusterEntry *e = cluster_kernel_at(i);
                    if (e->logn == v[0] && e->log1 == v[1] && e->loge == v[2] && e->r == v[3] && e->lay == v[4]) {
                        c.cl = e;
                        ok = true;
                    }
                }
        }
        if (ok) g_tune_cache[std::make_tuple((int64_t)n, (int64_t)batch, lay, dir, prec)] = c;
    }
    fclose(f);
}

void append_tune_file(const std::tuple<int64_t, int64_t, int, int, int> &key, const Choice &c, int npasses) {
    const char *path = getenv("FFTC_TUNE_CACHE");
    if (!path || !*path) return;
    char head[384];
    snprintf(head, sizeof(head), "plan %s|%lld %lld %d %d %d", device_name().c_str(), (long long)std::get<0>(key),
             (long long)std::get<1>(key), std::get<2>(key), std::get<3>(key), std::get<4>(key));
    std::string line = head;
    if (c.cl) {
        char b[96];
        snprintf(b, sizeof(b), " C %d %d %d %d %d", c.cl->logn, c.cl->log1, c.cl->loge, c.cl->r, c.cl->lay);
        line += b;
    } else if (npasses == 2) {
        char b[64];
        snprintf(b, sizeof(b), " F %d %d", c.logm, c.pf1);
        line += b;
        put_kernel(line, c.k1);
        put_kernel(line, c.k2);
    } else {
        line += " S";
        put_kernel(line, c.k1);
    }
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s\n", line.c_str());
    fclose(f);
}

struct Scratch {
    void *in = nullptr, *out = nullptr;
    void *ws = nullptr;  // the four-step workspace: the plan's, or a scratch one when it has none
    bool own_ws = false;
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    ~Scratch() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
        if (st) cudaStreamDestroy(st);
        if (in) cudaFree(in);
        if (out) cudaFree(out);
        if (own_ws && ws) cudaFree(ws);
    }
};

// stage tables of (logl, loge), uploaded once per plan (NULL for a single-stage line,
// which reads none); false if the upload failed
bool tables_for(fftc_plan_s *p, std::map<std::pair<int, int>, const float2 *> &cache, int logl, int loge,
                const float2 **out) {
    auto it = cache.find({logl, loge});
    if (it != cache.end()) {
        *out = it->second;
        return true;
    }
    std::vector<float2> tw;
    stage_twiddles(logl, loge, tw);
    void *d = nullptr;
    if (!tw.empty() && plan_upload(p, tw.data(), tw.size() * sizeof(float2), &d) != cudaSuccess) return false;
    cache[{logl, loge}] = (const float2 *)d;
    *out = (const float2 *)d;
    return true;
}

// mean milliseconds of one launch of `k` with `a`, or a negative value if it cannot run
float time_launch(const KernelEntry *k, const PassParams &a, Scratch &s, int reps) {
    if (k->prepare() != cudaSuccess) {
        cudaGetLastError();
        return -1.f;
    }
    if (k->launch(a, s.st) != cudaSuccess || cudaStreamSynchronize(s.st) != cudaSuccess) {
        cudaGetLastError();
        return -1.f;
    }
    cudaEventRecord(s.a, s.st);
    for (int i = 0; i < reps; ++i) k->launch(a, s.st);
    cudaEventRecord(s.b, s.st);
    if (cudaEventSynchronize(s.b) != cudaSuccess) return -1.f;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, s.a, s.b);
    return ms / reps;
}

fftc_status apply(fftc_plan_s *p, const Choice &c, std::map<std::pair<int, int>, const float2 *> &tabs) {
    if (c.cl) {  // one HBM round trip on a cluster: no workspace
        if (p->cluster != c.cl) {
            fftc_status st = cluster_setup(p, c.cl);
            if (st != FFTC_OK) return st;
        }
        if (p->workspace) plan_release(p, p->workspace);
        p->workspace = nullptr;
        return FFTC_OK;
    }
    if (p->cluster) {  // back from the cluster pass to the two four-step passes
        const int lay = p->layout == FFTC_LAYOUT_SPLIT ? LAYOUT_SPLIT : LAYOUT_IL;
        void *d = nullptr;
        if (plan_alloc(p, (size_t)p->total_elems * sizeof(float2), &d) != cudaSuccess) return FFTC_ERR_ALLOC;
        p->workspace = (float2 *)d;
        p->cluster = nullptr;
        p->npasses = 2;
        PassPlan &q0 = p->pass[0], &q1 = p->pass[1];
        q0.kind = KIND_COLS;
        q0.lin = lay;
        q0.lout = LAYOUT_IL;
        q0.logl = -1;  // forces the split's tables and parameters below
        q1.kind = KIND_ROWST;
        q1.lin = LAYOUT_IL;
        q1.lout = lay;
    }
    const float2 *t0 = nullptr, *t1 = nullptr;
    if (!tables_for(p, tabs, c.k1->logl, c.k1->loge, &t0)) return FFTC_ERR_ALLOC;
    if (p->npasses == 2 && !tables_for(p, tabs, c.k2->logl, c.k2->loge, &t1)) return FFTC_ERR_ALLOC;
    if (c.k1->prepare() != cudaSuccess || (p->npasses == 2 && c.k2->prepare() != cudaSuccess)) return FFTC_ERR_CUDA;
    PassPlan &p0 = p->pass[0];
    if (p->npasses == 2 && c.logm != p0.logl) {  // another split: its diagonal and pass shapes
        if (p->tw2_full) {
            float2 *d = nullptr;
            fftc_status st = upload_full_diagonal(p, c.logm, &d);
            if (st != FFTC_OK) return st;
            plan_release(p, p->tw2_full);
            p->tw2_full = d;
        }
        four_step_params(p, c.logm, p0.base, p->pass[1].base);
        p0.logl = c.logm;
        p->pass[1].logl = p->logn - c.logm;
    }
    p0.k = c.k1;
    p0.loge = c.k1->loge;
    p0.lines = c.k1->lines;
    p0.tw = const_cast<float2 *>(t0);
    p0.base.tw = t0;
    if (p->npasses == 2) {
        p0.base.pf_tiles = c.pf1;
        PassPlan &p1 = p->pass[1];
        p1.k = c.k2;
        p1.loge = c.k2->loge;
        p1.lines = c.k2->lines;
        p1.tw = const_cast<float2 *>(t1);
        p1.base.tw = t1;
    }
    return FFTC_OK;
}

// registry tag of the plan's kernels: 0 (FP32 on CUDA cores) or the tensor-core mode
int prec_of(const fftc_plan_s *p) { return p->precision == FFTC_FP32 ? 0 : (int)p->precision; }

// time of the cluster single pass `ce` on the plan's shape (its own diagonal and tables)
float time_cluster(fftc_plan_s *p, const ClusterEntry *ce, Scratch &s, int reps,
                   std::map<std::pair<int, int>, const float2 *> &tabs, fftc_status *err) {
    if (ce->prepare() != cudaSuccess) {
        cudaGetLastError();
        return -1.f;
    }
    float2 *diag = nullptr;
    if ((*err = upload_full_diagonal(p, ce->log1, &diag)) != FFTC_OK) return -1.f;
    const int log2 = p->logn - ce->log1, inv = p->direction == FFTC_INVERSE ? 1 : 0;
    int logr = 0;
    while ((1 << logr) < ce->r) ++logr;
    PassParams a, b;
    four_step_params(p, ce->log1, a, b);
    a.tw2_full = diag;
    a.cl_log_rows = ce->log1 - logr;
    a.in = (const float *)s.in;
    a.conj_in = inv;
    b.out = (float *)s.out;
    b.conj_out = inv;
    float ms = -1.f;
    if (!tables_for(p, tabs, ce->log1, ce->loge, &a.tw) || !tables_for(p, tabs, log2, ce->loge, &b.tw)) {
        *err = FFTC_ERR_ALLOC;
    } else if (ce->launch(a, b, p->batch, s.st) == cudaSuccess && cudaStreamSynchronize(s.st) == cudaSuccess) {
        cudaEventRecord(s.a, s.st);
        for (int i = 0; i < reps; ++i) ce->launch(a, b, p->batch, s.st);
        cudaEventRecord(s.b, s.st);
        if (cudaEventSynchronize(s.b) == cudaSuccess) {
            cudaEventElapsedTime(&ms, s.a, s.b);
            ms /= reps;
        }
    } else {
        cudaGetLastError();
    }
    plan_release(p, diag);
    return ms;
}

// fastest pass-1 and pass-2 kernels of one four-step split, with their summed time
float time_split(fftc_plan_s *p, int logm, const float2 *diag, Scratch &s, int reps,
                 std::map<std::pair<int, int>, const float2 *> &tabs, Choice *out, fftc_status *err) {
    const int lay = p->layout == FFTC_LAYOUT_SPLIT ? LAYOUT_SPLIT : LAYOUT_IL;
    const int logk = p->logn - logm, inv = p->direction == FFTC_INVERSE ? 1 : 0;
    PassParams a0, b0;
    four_step_params(p, logm, a0, b0);
    a0.tw2_full = diag;
    float t1 = 1e30f, t2 = 1e30f;
    Choice c;
    c.logm = logm;
    for (int i = 0; i < kernel_count(); ++i) {
        const KernelEntry *e = kernel_at(i);
        if (e->prec != prec_of(p)) continue;
        if (e->kind == KIND_COLS && e->logl == logm && e->lin == lay && e->lout == LAYOUT_IL &&
            (e->logx == 0 || e->logx == logk)) {
            for (int pf : {0, -1}) {
                if (pf && e->pipe) continue;  // the prefetch belongs to the plain kernel
                PassParams a = a0;
                if (!tables_for(p, tabs, e->logl, e->loge, &a.tw)) {
                    *err = FFTC_ERR_ALLOC;
                    return -1.f;
                }
                a.pf_tiles = pf;
                a.in = (const float *)s.in;
                a.out = (float *)s.ws;
                a.conj_in = inv;
                const float t = time_launch(e, a, s, reps);
                if (t > 0.f && t < t1) {
                    t1 = t;
                    c.k1 = e;
                    c.pf1 = pf;
                }
            }
        } else if (e->kind == KIND_ROWST && e->logl == logk && e->lin == LAYOUT_IL && e->lout == lay &&
                   (e->logx == 0 || e->logx == logm)) {
            PassParams b = b0;
            if (!tables_for(p, tabs, e->logl, e->loge, &b.tw)) {
                *err = FFTC_ERR_ALLOC;
                return -1.f;
            }
            b.in = (const float *)s.ws;
            b.out = (float *)s.out;
            b.conj_out = inv;
            const float t = time_launch(e, b, s, reps);
            if (t > 0.f && t < t2) {
                t2 = t;
                c.k2 = e;
            }
        }
    }
    if (!c.k1 || !c.k2) return -1.f;
    *out = c;
    return t1 + t2;
}

}  // namespace

fftc_status plan_tune(fftc_plan_s *p, int reps) {
    if (p->batch == 0) return FFTC_OK;
    if (p->mixed) return mixed_tune(p, reps);
    if (p->nd) return nd_tune(p, reps);
    if (p->uneven || p->fs || p->three) return FFTC_OK;
    if (reps < 1) reps = 1;
    const int lay = p->layout == FFTC_LAYOUT_SPLIT ? LAYOUT_SPLIT : LAYOUT_IL;
    const auto key = std::make_tuple(p->n, p->batch, (int)p->layout, (int)p->direction, (int)p->precision);
    std::map<std::pair<int, int>, const float2 *> tabs;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        if (!g_tune_file_read) {
            read_tune_file();
            g_tune_file_read = true;
        }
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) return apply(p, it->second, tabs);
    }
    Scratch s;
    const size_t bytes = (size_t)p->total_elems * 8;
    if (cudaMalloc(&s.in, bytes) != cudaSuccess || cudaMalloc(&s.out, bytes) != cudaSuccess) return FFTC_ERR_ALLOC;
    if (cudaMemset(s.in, 0, bytes) != cudaSuccess || cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&s.a) != cudaSuccess || cudaEventCreate(&s.b) != cudaSuccess)
        return FFTC_ERR_CUDA;
    const int inv = p->direction == FFTC_INVERSE ? 1 : 0;
    Choice best;
    best.logm = p->pass[0].logl;
    best.k1 = p->pass[0].k;
    best.k2 = p->npasses == 2 ? p->pass[1].k : nullptr;
    best.pf1 = p->pass[0].base.pf_tiles;
    best.cl = p->cluster;  // the plan as built, unless a candidate is faster
    const PassPlan &p0 = p->pass[0];
    if (p->npasses == 1 && !p->cluster) {
        float t1 = 1e30f;
        for (int i = 0; i < kernel_count(); ++i) {
            const KernelEntry *e = kernel_at(i);
            if (e->prec != prec_of(p) || e->kind != KIND_ROWS || e->logl != p0.logl || e->lin != lay || e->lout != lay)
                continue;
            PassParams a = p0.base;
            if (!tables_for(p, tabs, e->logl, e->loge, &a.tw)) return FFTC_ERR_ALLOC;
            a.in = (const float *)s.in;
            a.out = (float *)s.out;
            a.conj_in = a.conj_out = inv;
            const float t = time_launch(e, a, s, reps);
            if (t > 0.f && t < t1) {
                t1 = t;
                best.k1 = e;
            }
        }
    } else {
        if (p->workspace) {
            s.ws = p->workspace;
        } else {
            if (cudaMalloc(&s.ws, bytes) != cudaSuccess) return FFTC_ERR_ALLOC;
            s.own_ws = true;
        }
        // every split M K whose factors have compiled kernels (columns 2^6..2^12, rows 2^7..2^12)
        float tbest = 1e30f;
        for (int logm = 6; logm <= 12; ++logm) {
            const int logk = p->logn - logm;
            if (logk < 7 || logk > 12) continue;
            float2 *diag = nullptr;
            if (p->logn <= 20) {  // the whole diagonal of this split
                if (logm == p0.logl && p->tw2_full && !p->cluster) {
                    diag = p->tw2_full;
                } else {
                    fftc_status st = upload_full_diagonal(p, logm, &diag);
                    if (st != FFTC_OK) return st;
                }
            }
            Choice c;
            fftc_status err = FFTC_OK;
            const float t = time_split(p, logm, diag, s, reps, tabs, &c, &err);
            if (diag && diag != p->tw2_full) plan_release(p, diag);
            if (err != FFTC_OK) return err;
            if (t > 0.f && t < tbest) {
                tbest = t;
                best = c;
            }
        }
        // one HBM round trip on a thread-block cluster, every compiled shape for n and layout
        for (int i = 0; i < cluster_kernel_count() && p->precision == FFTC_FP32; ++i) {
            const ClusterEntry *ce = cluster_kernel_at(i);
            if (ce->logn != p->logn || ce->lay != lay) continue;
            fftc_status err = FFTC_OK;
            const float t = time_cluster(p, ce, s, reps, tabs, &err);
            if (err != FFTC_OK) return err;
            if (t > 0.f && t < tbest) {
                tbest = t;
                best = Choice();
                best.cl = ce;
            }
        }
    }
    if (!best.cl && (!best.k1 || ((p->npasses == 2 || p->cluster) && !best.k2))) return FFTC_ERR_UNSUPPORTED_SIZE;
    const fftc_status st = apply(p, best, tabs);
    if (st != FFTC_OK) return st;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
    append_tune_file(key, best, p->npasses);
    return FFTC_OK;
}

}  // namespace fftc

// Host side of the mixed-radix path (n = 2^a 3^b 5^c 7^d, not a power of two): radix
// factorisation, single pass up to kMixedSinglePass elements, Eq. 1 once at the HBM level
// (n = M K, both factors at most kMixedSinglePass) above, FP64-built stage tables and
// inter-pass diagonal, and the launches (kernels in fftc_mixed.cuh).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "fftc_mixed.cuh"
#include "fftc_mixed_ct.cuh"
#include "fftc_plan.h"

namespace fftc {

static const int kMixedSinglePass = 8192;  // longest FP32 line one CTA transforms (2 x 64 KB)
static const int kMixedTile = 4096;        // FP32 elements per CTA tile for shorter lines
static const int kMixedSinglePass64 = 4096;  // the same for FP64 (16-byte elements)
static const int kMixedTile64 = 2048;

extern const MixedKernel kMixedRowsF32[2][2], kMixedRowsF64[2][2], kMixedColsIlF32[2], kMixedColsIlF64[2],
    kMixedColsSplitF32[2][2], kMixedColsSplitF64[2][2], kMixedRowsTF32[2][2], kMixedRowsTF64[2][2];

struct MixedPass {
    MixedArgs args;
    MixedKernel kernel = nullptr;
    int smem = 0, threads = 256;
    int64_t blocks = 0;
};

static bool is_fp64(const fftc_plan_s *p) { return p->precision == FFTC_FP64; }

struct MixedState {
    int npasses = 0;
    int64_t m = 0;  // the split n = M K of a two-pass plan
    MixedPass pass[2];
};

bool mixed_supported(int64_t n) {
    if (n < 2 || n > (int64_t(1) << 24)) return false;
    int64_t m = n;
    for (int p : {2, 3, 5, 7})
        while (m % p == 0) m /= p;
    return m == 1;
}

// The first factor M of the split n = M K used above one CTA's line (M closest to sqrt n
// with both factors at most that line), 0 when n has none, n itself for one pass.
int64_t mixed_split(int64_t n, bool fp64) {
    const int64_t single = fp64 ? kMixedSinglePass64 : kMixedSinglePass;
    if (n <= single) return n;
    int64_t M = 0;
    for (int64_t m = 2; m <= single; ++m)
        if (n % m == 0 && n / m <= single &&
            (M == 0 || std::llabs((long long)(m * m - n)) < std::llabs((long long)(M * M - n))))
            M = m;
    return M;
}

// Radices of a line in stage order, at most 16 (a butterfly's values stay in registers):
// 3 x 5 = 15 and 3 x 3 = 9 first, then the remaining 3, 5, 7, the power-of-two remainder
// (2, 4 or 8), folded into one leftover odd factor where the product stays <= 16 (6, 10,
// 14, 12), and the radix-16 stages last, where Ns is largest.
static int getenv_int(const char *name, int dflt) {
    const char *v = getenv(name);
    return (v && *v) ? atoi(v) : dflt;
}

static std::vector<int> mixed_radices(int64_t L) {
    int e[8] = {0};
    int64_t m = L;
    for (int p : {2, 3, 5, 7})
        while (m % p == 0) {
            m /= p;
            ++e[p];
        }
    std::vector<int> odd;
    while (e[3] >= 1 && e[5] >= 1) {
        odd.push_back(15);
        --e[3];
        --e[5];
    }
    while (e[3] >= 2) {
        odd.push_back(9);
        e[3] -= 2;
    }
    for (int p : {7, 5, 3})
        for (; e[p] > 0; --e[p]) odd.push_back(p);
    int rem = 1 << (e[2] % 4);
    for (size_t i = 0; i < odd.size() && rem > 1; ++i)
        if ((odd[i] == 3 || odd[i] == 5 || odd[i] == 7) && odd[i] * rem <= 16) {
            odd[i] *= rem;
            rem = 1;
        }
    std::vector<int> r = odd;
    if (rem > 1) r.push_back(rem);
    for (int i = 0; i < e[2] / 4; ++i) r.push_back(16);
    return r;
}

static FastDiv make_div(uint32_t d) {
    FastDiv f;
    f.d = d;
    uint32_t l = 0;
    while ((uint64_t(1) << l) < d) ++l;
    f.l = l;
    f.m = (uint32_t)(((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1);
    return f;
}

// the division must be exact for every dividend below `limit` (< 2^31): check the ends
// of the range and a spread of points in between
static bool check_div(const FastDiv &f, uint64_t limit) {
    if (limit > (uint64_t(1) << 31)) return false;
    auto ok = [&](uint64_t n) { return fdiv((uint32_t)n, f) == (uint32_t)(n / f.d); };
    for (uint64_t n = 0; n < std::min<uint64_t>(limit, 4096); ++n)
        if (!ok(n)) return false;
    for (uint64_t n = limit > 4096 ? limit - 4096 : 0; n < limit; ++n)
        if (!ok(n)) return false;
    for (uint64_t n = 0; n < limit; n += 1 + limit / 65536)
        if (!ok(n)) return false;
    return true;
}

// the compiled variant for (kind, layouts, CTA size, element type); NULL if none
static MixedKernel mixed_kernel(int kind, int lin, int lout, int nt, bool fp64) {
    const int w = nt == 512 ? 1 : 0;
    if (kind == KIND_ROWS) return (fp64 ? kMixedRowsF64 : kMixedRowsF32)[lin == LAYOUT_IL ? 0 : 1][w];
    if (kind == KIND_COLS) {
        if (lin == LAYOUT_IL) return lout == LAYOUT_IL ? (fp64 ? kMixedColsIlF64 : kMixedColsIlF32)[w] : nullptr;
        return (fp64 ? kMixedColsSplitF64 : kMixedColsSplitF32)[lout == LAYOUT_IL ? 0 : 1][w];
    }
    if (kind == KIND_ROWST && lin == LAYOUT_IL) return (fp64 ? kMixedRowsTF64 : kMixedRowsTF32)[lout == LAYOUT_IL ? 0 : 1][w];
    return nullptr;
}

// stage tables of a line: stage s holds w_{Ns r}^{t k} at (t - 1) Ns + k (t < r, k < Ns)
static fftc_status mixed_pass_setup(fftc_plan_s *p, MixedPass &mp, int64_t L, int C, int kind, int lin, int lout,
                                    int64_t lpt) {
    const std::vector<int> rad = mixed_radices(L);
    if (rad.empty() || (int)rad.size() > kMixedMaxStages) return FFTC_ERR_UNSUPPORTED_SIZE;
    const bool fp64 = is_fp64(p);
    MixedArgs &a = mp.args;
    a.L = (int32_t)L;
    a.C = C;
    a.nst = (int32_t)rad.size();
    // single pass: lines back to back (flat copies); four-step: an odd pitch for column access
    a.pitch = (int32_t)L + (kind != KIND_ROWS && C > 1 && (L & 1) == 0 ? 1 : 0);
    a.lpt = (int32_t)lpt;
    a.flat = kind == KIND_ROWS && lin == LAYOUT_SPLIT && !fp64 && L <= 128;  // measured crossover
    std::vector<float2> tw;     // FP32 tables
    std::vector<double2> tw64;  // FP64 tables (the same entries, unrounded)
    int64_t ns = 1;
    for (int s = 0; s < a.nst; ++s) {
        const int r = rad[(size_t)s];
        a.radix[s] = (int8_t)r;
        a.ns[s] = (int32_t)ns;
        a.tw_off[s] = (int32_t)(fp64 ? tw64.size() : tw.size());
        a.div_lr[s] = make_div((uint32_t)(L / r));
        a.div_ns[s] = make_div((uint32_t)ns);
        if (!check_div(a.div_lr[s], (uint64_t)C * L) || !check_div(a.div_ns[s], (uint64_t)L))
            return FFTC_ERR_UNSUPPORTED_SIZE;
        if (ns > 1)
            for (int t = 1; t < r; ++t)
                for (int64_t k = 0; k < ns; ++k) {
                    double c, sn;
                    unit_root((int64_t)t * k, ns * r, &c, &sn);
                    if (fp64) tw64.push_back(make_double2(c, -sn));
                    else tw.push_back(make_float2((float)c, (float)-sn));
                }
        ns *= r;
    }
    a.div_L = make_div((uint32_t)L);
    a.div_C = make_div((uint32_t)C);
    a.div_lpt = make_div((uint32_t)lpt);
    const uint64_t tile = (uint64_t)C * L;
    if (!check_div(a.div_L, tile) || !check_div(a.div_C, tile) ||
        !check_div(a.div_lpt, (uint64_t)a.p.total_lines + (uint64_t)C))
        return FFTC_ERR_UNSUPPORTED_SIZE;
    if (!tw.empty() || !tw64.empty()) {
        void *d = nullptr;
        const cudaError_t e = fp64 ? plan_upload(p, tw64.data(), tw64.size() * sizeof(double2), &d)
                                   : plan_upload(p, tw.data(), tw.size() * sizeof(float2), &d);
        if (e != cudaSuccess) return FFTC_ERR_ALLOC;
        a.p.tw = (const float2 *)d;  // reinterpreted as double2 by the FP64 kernels
    }
    // 512 threads for tiles of more than 4096 elements (one or two CTAs per SM)
    const int nt = tile > 4096 ? 512 : 256;
    mp.threads = nt;
    mp.kernel = mixed_kernel(kind, lin, lout, nt, fp64);
    if (!mp.kernel) return FFTC_ERR_UNSUPPORTED_SIZE;
    // the per-length kernel of this exact shape, where one is compiled (FP32)
    if (!fp64 && getenv_int("FFTC_MIXED_CT", 1)) {
        const MixedCtEntry *ct = find_mixed_ct(kind, lin, lout, nt, (int)L, C, a.pitch, a.nst, a.radix);
        if (ct) mp.kernel = ct->kernel;
    }
    mp.smem = (((C * a.pitch + 1) & ~1) + C * a.pitch) * (int)(fp64 ? sizeof(double2) : sizeof(float2));
    if (mp.smem > 48 * 1024) {
        // the dynamic shared memory of one kernel differs from plan to plan: allow the
        // device's maximum once (a smaller limit set for a later plan would break an
        // earlier one); the launch's own size still sets the occupancy
        int dev = 0, cap = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            return FFTC_ERR_CUDA;
        if (mp.smem > cap) return FFTC_ERR_UNSUPPORTED_SIZE;
        if (cudaFuncSetAttribute((const void *)mp.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, cap) !=
            cudaSuccess)
            return FFTC_ERR_CUDA;
    }
    mp.blocks = (a.p.total_lines + C - 1) / C;
    return FFTC_OK;
}

static int mixed_lines(int64_t L, bool fp64 = false) {
    return (int)std::max<int64_t>(1, (fp64 ? kMixedTile64 : kMixedTile) / L);
}

fftc_status mixed_build(fftc_plan_s *p) {
    if (p->precision != FFTC_FP32 && p->precision != FFTC_FP64) return FFTC_ERR_UNSUPPORTED_SIZE;
    const bool fp64 = is_fp64(p);
    const int64_t single = fp64 ? kMixedSinglePass64 : kMixedSinglePass;
    MixedState *ms = new (std::nothrow) MixedState();
    if (!ms) return FFTC_ERR_ALLOC;
    p->mixed = ms;
    const int64_t n = p->n, B = p->batch;
    const int lay = p->layout == FFTC_LAYOUT_SPLIT ? LAYOUT_SPLIT : LAYOUT_IL;
    const int64_t plane = lay == LAYOUT_SPLIT ? n * B : 0;
    p->total_elems = n * B;
    void *d = nullptr;
    if (plan_alloc(p, 16, &d) != cudaSuccess) return FFTC_ERR_ALLOC;
    p->d_err = (int *)d;
    if (cudaMemset(p->d_err, 0, 16) != cudaSuccess) return FFTC_ERR_CUDA;
    if (n <= single) {
        ms->npasses = p->npasses = 1;
        MixedPass &mp = ms->pass[0];
        PassParams &b = mp.args.p;
        memset(&b, 0, sizeof(b));
        b.err = p->d_err;
        b.in_plane = b.out_plane = plane;
        b.total_lines = B;
        b.in_tr = b.out_tr = n;
        b.in_elem = b.out_elem = 1;
        // a multiple of 4 lines per tile when there are several, so every tile starts 16-byte
        // aligned in both layouts
        const int C = mixed_lines(n, fp64);
        return mixed_pass_setup(p, mp, n, C >= 4 ? C / 4 * 4 : C, KIND_ROWS, lay, lay, 1);
    }
    // n = M K with both factors at most one CTA's line, M as close to sqrt(n) as possible
    // unless measure-mode planning chose another split
    const bool forced = p->force_m > 1 && n % p->force_m == 0 && p->force_m <= single && n / p->force_m <= single;
    const int64_t M = forced ? p->force_m : mixed_split(n, fp64);
    if (M == 0) return FFTC_ERR_UNSUPPORTED_SIZE;
    const int64_t K = n / M;
    ms->m = M;
    ms->npasses = p->npasses = 2;
    const size_t esz = fp64 ? sizeof(double2) : sizeof(float2);
    if (plan_alloc(p, (size_t)(n * B) * esz, &d) != cudaSuccess) return FFTC_ERR_ALLOC;
    p->workspace = (float2 *)d;
    {  // the inter-pass diagonal D of Eq. 1 in pass-1 order: entry t' K + b = w_N^(b t')
        std::vector<float2> full(fp64 ? 0 : (size_t)n);
        std::vector<double2> full64(fp64 ? (size_t)n : 0);
        for (int64_t tp = 0; tp < M; ++tp)
            for (int64_t b = 0; b < K; ++b) {
                double c, s;
                unit_root(tp * b, n, &c, &s);
                if (fp64) full64[(size_t)(tp * K + b)] = make_double2(c, -s);
                else full[(size_t)(tp * K + b)] = make_float2((float)c, (float)-s);
            }
        const cudaError_t e = fp64 ? plan_upload(p, full64.data(), full64.size() * sizeof(double2), &d)
                                   : plan_upload(p, full.data(), full.size() * sizeof(float2), &d);
        if (e != cudaSuccess) return FFTC_ERR_ALLOC;
        p->tw2_full = (float2 *)d;
    }
    {  // pass 1: K columns of length M at stride K, times the diagonal, into the workspace
        MixedPass &mp = ms->pass[0];
        PassParams &b = mp.args.p;
        memset(&b, 0, sizeof(b));
        b.err = p->d_err;
        b.in_plane = plane;
        b.total_lines = B * K;
        b.in_tr = b.out_tr = n;
        b.in_line = b.out_line = 1;
        b.in_elem = b.out_elem = K;
        b.tw2_full = p->tw2_full;
        fftc_status s = mixed_pass_setup(p, mp, M, (int)std::min<int64_t>(K, mixed_lines(M, fp64)), KIND_COLS,
                                         lay, LAYOUT_IL, K);
        if (s != FFTC_OK) return s;
    }
    {  // pass 2: M rows of length K, stored transposed (output k1 + M k2)
        MixedPass &mp = ms->pass[1];
        PassParams &b = mp.args.p;
        memset(&b, 0, sizeof(b));
        b.err = p->d_err;
        b.out_plane = plane;
        b.total_lines = B * M;
        b.in_tr = b.out_tr = n;
        b.in_line = K;
        b.in_elem = 1;
        b.out_line = 1;
        b.out_elem = M;
        return mixed_pass_setup(p, mp, K, (int)std::min<int64_t>(M, mixed_lines(K, fp64)), KIND_ROWST, LAYOUT_IL,
                                lay, M);
    }
}

static cudaError_t mixed_launch(const MixedPass &mp, const MixedArgs &a, cudaStream_t st) {
    if (mp.blocks <= 0) return cudaSuccess;
    if (mp.blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
    void *kargs[] = {(void *)&a};
    return cudaLaunchKernel((const void *)mp.kernel, dim3((unsigned)mp.blocks), dim3(mp.threads), kargs,
                            (size_t)mp.smem, st);
}

fftc_status mixed_run(fftc_plan_s *p, const void *in, void *out, const float *post_h, float post_scale,
                      cudaStream_t st) {
    const MixedState *ms = p->mixed;
    const int inv = p->direction == FFTC_INVERSE ? 1 : 0;
    if (post_h && p->precision != FFTC_FP32) return FFTC_ERR_INVALID_VALUE;
    if (ms->npasses == 1) {
        MixedArgs a = ms->pass[0].args;
        a.p.in = (const float *)in;
        a.p.out = (float *)out;
        a.p.conj_in = a.p.conj_out = inv;
        a.p.post_h = post_h;
        a.p.post_scale = post_scale;
        a.p.post_line_mul = 0;  // frequency = position in the line
        a.p.post_elem_mul = 1;
        return mixed_launch(ms->pass[0], a, st) == cudaSuccess ? FFTC_OK : FFTC_ERR_CUDA;
    }
    MixedArgs a = ms->pass[0].args;
    a.p.in = (const float *)in;
    a.p.out = (float *)p->workspace;
    a.p.conj_in = inv;
    if (mixed_launch(ms->pass[0], a, st) != cudaSuccess) return FFTC_ERR_CUDA;
    MixedArgs b = ms->pass[1].args;
    b.p.in = (const float *)p->workspace;
    b.p.out = (float *)out;
    b.p.conj_out = inv;
    b.p.post_h = post_h;  // pass 2 writes frequency k1 + M k2 (line k1, position k2)
    b.p.post_scale = post_scale;
    b.p.post_line_mul = 1;
    b.p.post_elem_mul = ms->pass[0].args.L;
    return mixed_launch(ms->pass[1], b, st) == cudaSuccess ? FFTC_OK : FFTC_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Multidimensional transforms over [batch][d0]...[d_{r-1}] (rank 2 or 3): the DFT along
// the contiguous last axis by a one-dimensional plan, then along every other axis a is a
// strided pass of the column kind in place: line = (outer index, position l inside the
// block of the later axes S = d_{a+1} ... d_{r-1}), element stride S, no inter-pass twiddle.
// This is the (F (x) I)(I (x) F) form of Section 3 with both factors whole transforms.
// ---------------------------------------------------------------------------

struct NdState {
    fftc_plan_s *rows = nullptr;
    int naxes = 0;
    MixedPass axes[2];
    // power-of-two axes of 64..1024 points: the compiled column pass
    // (k_pass, runtime element stride) instead of the runtime-radix kernel
    const KernelEntry *fast[2] = {nullptr, nullptr};
    PassParams fastp[2];
};

// compiled column-pass shape for a strided power-of-two axis (log2 length, log2 elements
// per thread, columns per tile), or false
static bool nd_fast_shape(int64_t L, int *logl, int *loge, int *lines) {
    if (L < 64 || L > 1024 || (L & (L - 1)) != 0) return false;
    int l = 0;
    while ((int64_t(1) << l) < L) ++l;
    *logl = l;
    *loge = l == 10 ? 5 : 4;
    *lines = l == 10 ? 8 : 16;
    return true;
}

bool nd_axis_supported(int64_t d, bool fp64) {
    return d >= 2 && d <= (fp64 ? kMixedSinglePass64 : kMixedSinglePass) && (mixed_supported(d) || (d & (d - 1)) == 0);
}

fftc_status nd_build(fftc_plan_s *p, int rank, const int64_t *dims) {
    NdState *nd = new (std::nothrow) NdState();
    if (!nd) return FFTC_ERR_ALLOC;
    p->nd = nd;
    const int lay = p->layout == FFTC_LAYOUT_SPLIT ? LAYOUT_SPLIT : LAYOUT_IL;
    int64_t total = p->batch;
    for (int a = 0; a < rank; ++a) total *= dims[a];
    p->total_elems = total;
    void *d = nullptr;
    if (plan_alloc(p, 16, &d) != cudaSuccess) return FFTC_ERR_ALLOC;
    p->d_err = (int *)d;
    if (cudaMemset(p->d_err, 0, 16) != cudaSuccess) return FFTC_ERR_CUDA;
    // the last axis: a one-dimensional plan over batch * d0 ... d_{r-2} contiguous rows
    fftc_plan_s *r = new (std::nothrow) fftc_plan_s();
    if (!r) return FFTC_ERR_ALLOC;
    nd->rows = r;
    r->magic = p->magic;
    r->device = p->device;
    r->n = dims[rank - 1];
    r->logn = 0;
    while ((int64_t(1) << (r->logn + 1)) <= r->n) ++r->logn;
    r->batch = total / r->n;
    r->layout = p->layout;
    r->direction = p->direction;
    r->precision = p->precision;
    fftc_status st = plan_build(r);
    if (st != FFTC_OK) return st;
    const int64_t plane = lay == LAYOUT_SPLIT ? total : 0;
    for (int a = rank - 2; a >= 0; --a) {
        int64_t S = 1, outer = p->batch;
        for (int b = a + 1; b < rank; ++b) S *= dims[b];
        for (int b = 0; b < a; ++b) outer *= dims[b];
        const int64_t L = dims[a];
        const int ax = nd->naxes++;
        int logl = 0, loge = 0, lines = 0;
        if (!is_fp64(p) && (S & (S - 1)) == 0 && nd_fast_shape(L, &logl, &loge, &lines)) {
            const KernelEntry *k = find_kernel(KIND_COLS, logl, loge, lines, lay, lay, 0, 0);
            if (k) {
                PassParams &q = nd->fastp[ax];
                memset(&q, 0, sizeof(q));
                q.err = p->d_err;
                q.total_lines = outer * S;
                q.in_plane = q.out_plane = plane;
                int ls = 0;
                while ((int64_t(1) << ls) < S) ++ls;
                q.log_lpt = ls;
                q.in_tr = q.out_tr = L * S;
                q.in_line = q.out_line = 1;
                q.in_elem = q.out_elem = S;
                // prefetch the next wave's column bands into L2 (tiles inside one block only)
                q.pf_tiles = S >= lines ? -1 : 0;
                std::vector<float2> tw;
                stage_twiddles(logl, loge, tw);
                if (!tw.empty()) {
                    if (plan_upload(p, tw.data(), tw.size() * sizeof(float2), &d) != cudaSuccess) return FFTC_ERR_ALLOC;
                    q.tw = (const float2 *)d;
                }
                if (k->prepare() != cudaSuccess) return FFTC_ERR_CUDA;
                nd->fast[ax] = k;
                // the runtime-radix pass of the axis is built too: measure-mode planning
                // may prefer it
            }
        }
        MixedPass &mp = nd->axes[ax];
        PassParams &b = mp.args.p;
        memset(&b, 0, sizeof(b));
        b.err = p->d_err;
        b.in_plane = b.out_plane = plane;
        b.total_lines = outer * S;
        b.in_tr = b.out_tr = L * S;
        b.in_line = b.out_line = 1;
        b.in_elem = b.out_elem = S;
        const bool fp64 = is_fp64(p);
        if (b.total_lines + mixed_lines(L, fp64) >= (int64_t(1) << 31)) return FFTC_ERR_UNSUPPORTED_SIZE;
        st = mixed_pass_setup(p, mp, L, (int)std::min<int64_t>(S, mixed_lines(L, fp64)), KIND_COLS, lay, lay, S);
        if (st != FFTC_OK) return st;
    }
    p->npasses = r->npasses + nd->naxes;
    return FFTC_OK;
}

fftc_status nd_run(fftc_plan_s *p, const void *in, void *out, cudaStream_t st) {
    NdState *nd = p->nd;
    fftc_status s = plan_run(nd->rows, in, out, nullptr, 0.f, st);
    if (s != FFTC_OK) return s;
    const int inv = p->direction == FFTC_INVERSE ? 1 : 0;
    for (int i = 0; i < nd->naxes; ++i) {  // in place: a tile is read whole before it is written
        if (nd->fast[i]) {
            PassParams q = nd->fastp[i];
            q.in = (const float *)out;
            q.out = (float *)out;
            q.conj_in = q.conj_out = inv;
            if (nd->fast[i]->launch(q, st) != cudaSuccess) return FFTC_ERR_CUDA;
            continue;
        }
        MixedArgs a = nd->axes[i].args;
        a.p.in = (const float *)out;
        a.p.out = (float *)out;
        a.p.conj_in = a.p.conj_out = inv;
        if (mixed_launch(nd->axes[i], a, st) != cudaSuccess) return FFTC_ERR_CUDA;
    }
    return FFTC_OK;
}

void nd_free(fftc_plan_s *p) {
    if (!p->nd) return;
    if (p->nd->rows) {
        plan_destroy_extra(p->nd->rows);
        plan_free_device(p->nd->rows);
        delete p->nd->rows;
    }
    delete p->nd;
    p->nd = nullptr;
}

int mixed_radix_list(const fftc_plan_s *p, int *radices, int cap) {
    int cnt = 0;
    for (int i = 0; i < p->mixed->npasses; ++i) {
        const MixedArgs &a = p->mixed->pass[i].args;
        for (int s = 0; s < a.nst; ++s)
            if (cnt < cap) radices[cnt++] = a.radix[s];
    }
    return cnt;
}

void mixed_free(fftc_plan_s *p) {
    delete p->mixed;
    p->mixed = nullptr;
}

int64_t mixed_plan_split(const fftc_plan_s *p) {
    return (p->mixed && p->mixed->npasses == 2) ? p->mixed->m : p->n;
}

// ---------------------------------------------------------------------------
// measure-mode planning (the runtime decomposition search of Section 6)
// ---------------------------------------------------------------------------
namespace {

struct TuneBufs {
    void *in = nullptr, *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    ~TuneBufs() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
        if (st) cudaStreamDestroy(st);
        if (in) cudaFree(in);
        if (out) cudaFree(out);
    }
    bool init(size_t bytes) {
        return cudaMalloc(&in, bytes) == cudaSuccess && cudaMalloc(&out, bytes) == cudaSuccess &&
               cudaMemset(in, 0, bytes) == cudaSuccess &&
               cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
               cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess;
    }
    // mean milliseconds of `reps` runs of fn(stream) after one untimed run; < 0 on failure
    template <class F>
    float time(F fn, int reps) {
        if (!fn(st) || cudaStreamSynchronize(st) != cudaSuccess) {
            cudaGetLastError();
            return -1.f;
        }
        cudaEventRecord(a, st);
        for (int i = 0; i < reps; ++i) fn(st);
        cudaEventRecord(b, st);
        if (cudaEventSynchronize(b) != cudaSuccess) return -1.f;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        return ms / reps;
    }
};

std::mutex g_mixed_tune_mu;
std::map<std::tuple<int64_t, int64_t, int, int, int>, int64_t> g_mixed_tune_cache;

// a plan of p's shape built with the split n = m (n / m); nullptr on failure
fftc_plan_s *mixed_candidate(const fftc_plan_s *p, int64_t m) {
    fftc_plan_s *q = new (std::nothrow) fftc_plan_s();
    if (!q) return nullptr;
    q->magic = p->magic;
    q->device = p->device;
    q->n = p->n;
    q->logn = p->logn;
    q->batch = p->batch;
    q->layout = p->layout;
    q->direction = p->direction;
    q->precision = p->precision;
    q->force_m = m;
    if (plan_build(q) != FFTC_OK) {
        plan_destroy_extra(q);
        plan_free_device(q);
        delete q;
        return nullptr;
    }
    return q;
}

void drop_candidate(fftc_plan_s *q) {
    plan_destroy_extra(q);
    plan_free_device(q);
    delete q;
}

}  // namespace

fftc_status mixed_tune(fftc_plan_s *p, int reps) {
    if (!p->mixed || p->mixed->npasses != 2) return FFTC_OK;  // one pass: nothing to choose
    const bool fp64 = is_fp64(p);
    const int64_t n = p->n, single = fp64 ? kMixedSinglePass64 : kMixedSinglePass;
    const auto key = std::make_tuple(n, p->batch, (int)p->layout, (int)p->direction, (int)p->precision);
    int64_t best = 0;
    {
        std::lock_guard<std::mutex> lk(g_mixed_tune_mu);
        auto it = g_mixed_tune_cache.find(key);
        if (it != g_mixed_tune_cache.end()) best = it->second;
    }
    if (!best) {
        // candidate splits: divisors with both factors within one CTA's line, the six closest
        // to sqrt(n) (on a log scale)
        std::vector<int64_t> cand;
        for (int64_t m = 2; m <= single; ++m)
            if (n % m == 0 && n / m <= single) cand.push_back(m);
        const double c = 0.5 * std::log((double)n);
        std::sort(cand.begin(), cand.end(), [&](int64_t x, int64_t y) {
            return std::fabs(std::log((double)x) - c) < std::fabs(std::log((double)y) - c);
        });
        if (cand.size() > 6) cand.resize(6);
        TuneBufs tb;
        if (!tb.init((size_t)p->total_elems * (fp64 ? 16 : 8))) return FFTC_ERR_ALLOC;
        float tbest = 1e30f;
        for (int64_t m : cand) {
            fftc_plan_s *q = mixed_candidate(p, m);
            if (!q) continue;
            const float t = tb.time([&](cudaStream_t st) { return mixed_run(q, tb.in, tb.out, nullptr, 0.f, st) == FFTC_OK; },
                                    reps);
            drop_candidate(q);
            if (t > 0.f && t < tbest) {
                tbest = t;
                best = m;
            }
        }
        if (!best) return FFTC_OK;
        std::lock_guard<std::mutex> lk(g_mixed_tune_mu);
        g_mixed_tune_cache[key] = best;
    }
    if (best == p->mixed->m) return FFTC_OK;
    // rebuild the plan's device state with the chosen split (the handle and its timing
    // probe stay the same)
    fftc_plan_s *q = mixed_candidate(p, best);
    if (!q) return FFTC_ERR_ALLOC;
    mixed_free(p);
    plan_free_device(p);
    p->force_m = best;
    p->npasses = q->npasses;
    p->workspace = q->workspace;
    p->tw2_full = q->tw2_full;
    p->d_err = q->d_err;
    p->mixed = q->mixed;
    p->dev_allocs.swap(q->dev_allocs);
    q->mixed = nullptr;
    q->dev_allocs.clear();
    delete q;
    return FFTC_OK;
}

fftc_status nd_tune(fftc_plan_s *p, int reps) {
    NdState *nd = p->nd;
    if (!nd) return FFTC_OK;
    fftc_status s = plan_tune(nd->rows, reps);  // the last axis: a 1D plan
    if (s != FFTC_OK) return s;
    TuneBufs tb;
    bool ready = false;
    const int inv = p->direction == FFTC_INVERSE ? 1 : 0;
    for (int i = 0; i < nd->naxes; ++i) {
        if (!nd->fast[i]) continue;  // only the runtime-radix pass exists for this axis
        if (!ready) {
            if (!tb.init((size_t)p->total_elems * (is_fp64(p) ? 16 : 8))) return FFTC_ERR_ALLOC;
            ready = true;
        }
        const KernelEntry *k = nd->fast[i];
        const float tf = tb.time([&](cudaStream_t st) {
            PassParams q = nd->fastp[i];
            q.in = (const float *)tb.out;
            q.out = (float *)tb.out;
            q.conj_in = q.conj_out = inv;
            return k->launch(q, st) == cudaSuccess;
        }, reps);
        const float tm = tb.time([&](cudaStream_t st) {
            MixedArgs a = nd->axes[i].args;
            a.p.in = (const float *)tb.out;
            a.p.out = (float *)tb.out;
            a.p.conj_in = a.p.conj_out = inv;
            return mixed_launch(nd->axes[i], a, st) == cudaSuccess;
        }, reps);
        if (tm > 0.f && (tf <= 0.f || tm < tf)) nd->fast[i] = nullptr;
    }
    return FFTC_OK;
}

}  // namespace fftc

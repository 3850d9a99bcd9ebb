// Planner and executor of the FP32 power-of-two Stockham path (other lengths, FP64 and
// multidimensional plans are built in fftc_mixed.cu; plan_run dispatches to them).
//
// n <= 2^14: one fused pass (KIND_ROWS), each CTA transforming whole rows.
// n >  2^14: Eq. 1 applied once at the HBM level, n = M * K (four-step):
//   pass 1 (KIND_COLS):  K column FFTs of length M over x[t*K + b], times w_n^(b t'),
//                        written in place to the workspace z[t'*K + b];
//   pass 2 (KIND_ROWST): M row FFTs of length K over z[t'*K .. t'*K + K), written
//                        transposed to X[b'*M + t'] (natural order).
// Inverse transforms run the forward arithmetic on conj(x) and conjugate the
// result (F^H x = conj(F conj x)), so both directions share every kernel.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "fftc_plan.h"

namespace fftc {

static const int kMaxSinglePassLog = 14;
static const int kPassLines = 16;

static int env_int(const char *name, int dflt) {
    const char *v = getenv(name);
    if (!v || !*v) return dflt;
    return atoi(v);
}

bool choose_rows(int logn, int lin, int *loge, int *lines) {
    int e;
    if (logn <= 4) e = logn;
    else if (logn <= 8) e = 4;
    else if (logn == 12) e = 4;
    else e = 5;
    char name[64];
    snprintf(name, sizeof(name), "FFTC_TUNE_ROWS_E_%d", logn);
    e = env_int(name, e);
    if (e > logn) e = logn;
    const int tpl = 1 << (logn - e);
    int c = tpl >= 256 ? 1 : 256 / tpl;
    if (logn <= 4) c = 128;  // one thread per line: 128-line CTAs
    snprintf(name, sizeof(name), "FFTC_TUNE_ROWS_C_%d", logn);
    c = env_int(name, c);
    *loge = e;
    *lines = c;
    return find_kernel(KIND_ROWS, logn, e, c, lin, lin) != nullptr;
}

// Measured four-step shapes, n = M K (Eq. 1 at the memory level). Pass 1 reads bands of
// C1 adjacent columns (C1 * 8 bytes per row, the wider the better up to the tile budget of
// ~68 KB); pass 2 writes C2-element runs (narrower than 8 elements is slow, above all for
// the split layout). Pass-1 feed per layout: 0 = plain loads into registers, 5 = tensor-map
// boxes into one landing buffer refilled after the tile's last shared read; pass 2: 0 =
// plain, 6 = one bulk copy per tile into two landing buffers, early refill.
// A plain pass 1 also prefetches, into L2, the band of the tile launched one wave later
// (pf = 1) where that measured faster.
struct FourStepDefault {
    int logn, logm, e1, c1, p1_il, p1_split, pf, e2, c2, p2;
};
static const FourStepDefault kFourStepDefaults[] = {
    {14, 7, 4, 16, 0, 0, 1, 4, 16, 0}, {15, 7, 4, 16, 0, 5, 1, 4, 16, 0}, {16, 8, 4, 16, 0, 5, 1, 4, 16, 0},
    {17, 8, 4, 16, 0, 5, 1, 5, 8, 6},  {18, 8, 4, 32, 5, 5, 1, 5, 8, 6},  {19, 9, 4, 16, 0, 5, 1, 5, 8, 6},
    {20, 10, 5, 8, 0, 0, 0, 5, 8, 6},
    // above 2^20 a factor exceeds 2^10: column tiles of 16 lines of 2^10, 8 of 2^11 or 4 of
    // 2^12 with 16 elements per thread (1024 threads); pass 2 fed by one bulk copy per tile
    // except at 2^24 (the best of both layouts together)
    {21, 10, 4, 16, 0, 0, 0, 5, 8, 5}, {22, 11, 4, 8, 0, 0, 0, 5, 8, 5},  {23, 12, 4, 4, 0, 0, 0, 5, 8, 5},
    {24, 12, 4, 4, 0, 0, 0, 4, 4, 0},
};

FourStepChoice choose_four_step(int logn, int lay) {
    FourStepChoice c;
    const FourStepDefault *d = nullptr;
    for (const FourStepDefault &t : kFourStepDefaults)
        if (t.logn == logn) d = &t;
    const int m = env_int("FFTC_TUNE_FOURSTEP_LOGM", d ? d->logm : logn / 2), k = logn - m;
    const bool same = d && m == d->logm;  // the table row applies to this split
    c.logm = m;
    c.e1 = env_int("FFTC_TUNE_COLS_E", same ? d->e1 : (m >= 10 ? 5 : 4));
    c.e2 = env_int("FFTC_TUNE_ROWST_E", same ? d->e2 : (k >= 9 ? 5 : 4));
    if (c.e1 > m) c.e1 = m;
    if (c.e2 >= k) c.e2 = k - 1;
    c.c1 = env_int("FFTC_TUNE_COLS_C", same ? d->c1 : (m >= 12 ? 4 : (m >= 10 ? 8 : 16)));
    c.c2 = env_int("FFTC_TUNE_ROWST_C", same ? d->c2 : (k >= 12 ? 4 : (k >= 9 ? 8 : 16)));
    c.p1 = same ? (lay == LAYOUT_SPLIT ? d->p1_split : d->p1_il) : 0;
    c.p2 = same ? d->p2 : 0;
    c.pf = env_int("FFTC_PF", same ? d->pf : 0);
    // FFTC_PIPE4: bit 0 forces the pass-1 feed on or off (code FFTC_TUNE_P1_PIPE, default
    // tensor-map boxes with two buffers), bit 1 the pass-2 feed (FFTC_TUNE_P2_PIPE)
    const int force = env_int("FFTC_PIPE4", -1);
    if (force >= 0) {
        c.p1 = (force & 1) ? env_int("FFTC_TUNE_P1_PIPE", c.p1 ? c.p1 : 2) : 0;
        c.p2 = (force & 2) ? env_int("FFTC_TUNE_P2_PIPE", c.p2 ? c.p2 : 2) : 0;
    }
    return c;
}

// Default pipelined single-pass kernel per size: elements per thread (log2), lines per
// tile, pipe code (landing buffers | 4 when the refill follows the last shared read).
struct PipeRowsDefault {
    int logn, loge, lines, code;
};
static const PipeRowsDefault kPipeRowsDefaults[] = {
    {9, 5, 8, 2}, {10, 5, 4, 2}, {11, 5, 2, 6}, {12, 5, 1, 5}, {13, 5, 1, 5}, {14, 5, 1, 5},
};
static const PipeRowsDefault *pipe_rows_default(int logn) {
    for (const PipeRowsDefault &d : kPipeRowsDefaults)
        if (d.logn == logn) return &d;
    return nullptr;
}

// smallest log2 n planned as three HBM passes by default: measured (n * batch = 2^26,
// forward) against the two-pass form, 2^24 1.08x (interleaved) and 1.32x (split) faster,
// 2^23 even, 2^21 and 2^22 0.62-0.76x (the middle pass runs once per transform)
static constexpr int kThreePassMinLog = 24;

// Elements per thread (log2) of the tensor-core single pass: 5 (radix-32 stages) at 2^13
// and 2^14, where it measured 12-16 % faster than radix-16 stages (one stage and one
// exchange fewer), else 4 (at 2^12 the radix-16 tiles keep three CTAs per SM and win);
// FFTC_TUNE_TC_E overrides it.
static int tc_rows_loge(int logn) { return (logn == 13 || logn == 14) ? 5 : 4; }

// bounded waits: FFTC_SPIN_LIMIT sets the poll limit of the pipelined kernels, and
// FFTC_TEST_UNREACHABLE_WAIT (a test hook) makes them issue no copy so every wait runs out
static void set_wait_hooks(PassParams &b) {
    b.spin_limit = env_int("FFTC_SPIN_LIMIT", 0);
    b.test_no_copy = env_int("FFTC_TEST_UNREACHABLE_WAIT", 0) ? 1 : 0;
}

static fftc_status upload_stage_tables(fftc_plan_s *p, PassPlan &pp) {
    std::vector<float2> tw;
    stage_twiddles(pp.logl, pp.loge, tw);
    void *d = nullptr;
    if (plan_upload(p, tw.data(), tw.size() * sizeof(float2), &d) != cudaSuccess) return FFTC_ERR_ALLOC;
    pp.tw = (float2 *)d;
    pp.base.tw = pp.tw;
    return FFTC_OK;
}

static fftc_status prepare(PassPlan &pp) {
    if (!pp.k) return FFTC_ERR_UNSUPPORTED_SIZE;
    if (pp.k->prepare() != cudaSuccess) return FFTC_ERR_CUDA;
    return FFTC_OK;
}

fftc_status upload_full_diagonal(fftc_plan_s *p, int logm, float2 **out) {
    const int64_t n = p->n, M = int64_t(1) << logm, K = n >> logm;
    std::vector<float2> full((size_t)n);
    for (int64_t tp = 0; tp < M; ++tp)
        for (int64_t b = 0; b < K; ++b) {
            double c, s;
            unit_root(tp * b, n, &c, &s);
            full[(size_t)(tp * K + b)] = make_float2((float)c, (float)-s);
        }
    void *d = nullptr;
    if (plan_upload(p, full.data(), full.size() * sizeof(float2), &d) != cudaSuccess) return FFTC_ERR_ALLOC;
    *out = (float2 *)d;
    return FFTC_OK;
}

void four_step_params(const fftc_plan_s *p, int logm, PassParams &a, PassParams &b) {
    const int64_t n = p->n, B = p->batch, M = int64_t(1) << logm, K = n >> logm;
    const int logk = p->logn - logm;
    const int64_t plane = p->layout == FFTC_LAYOUT_SPLIT ? n * B : 0;
    memset(&a, 0, sizeof(a));
    a.err = p->d_err;
    set_wait_hooks(a);
    a.in_plane = plane;
    a.out_plane = 0;
    a.total_lines = B * K;
    a.log_lpt = logk;
    a.in_tr = n;
    a.in_line = 1;
    a.in_elem = K;
    a.out_tr = n;
    a.out_line = 1;
    a.out_elem = K;
    a.tw2_lo = p->tw2_lo;
    a.tw2_hi = p->tw2_hi;
    a.tw2_full = p->tw2_full;
    a.log_n2 = p->logn;
    a.tw2_lo_bits = p->tw2_lo_bits;
    memset(&b, 0, sizeof(b));
    b.err = p->d_err;
    set_wait_hooks(b);
    b.in_plane = 0;
    b.out_plane = plane;
    b.total_lines = B * M;
    b.log_lpt = logm;
    b.in_tr = n;
    b.in_line = K;
    b.in_elem = 1;
    b.out_tr = n;
    b.out_line = 1;
    b.out_elem = M;
    b.post_line_mul = 1;
    b.post_elem_mul = M;
}

// FP64 table w_N^m for m < count, m scaled by `step` (m * step taken mod N), rounded once
static fftc_status upload_roots(fftc_plan_s *p, int64_t N, int64_t count, int64_t step, float2 **out) {
    std::vector<float2> t((size_t)count);
    for (int64_t m = 0; m < count; ++m) {
        double c, s;
        unit_root((m * step) % N, N, &c, &s);
        t[(size_t)m] = make_float2((float)c, (float)-s);
    }
    void *d = nullptr;
    if (plan_upload(p, t.data(), t.size() * sizeof(float2), &d) != cudaSuccess) return FFTC_ERR_ALLOC;
    *out = (float2 *)d;
    return FFTC_OK;
}

// Three HBM passes: Eq. 1 at the memory level twice, n = M K with K = P Q.
//   pass 1 (columns): column j2 < K of every transform, M points at stride K, times
//           w_n^(j2 k1), into ws1[b][k1][j2];
//   pass 2 (columns, launched once per transform b): inside each row k1 of ws1, column
//           j4 < Q, P points at stride Q, times w_K^(j4 k3), into ws2[b][k3][k1][j4];
//   pass 3 (rows stored transposed): row (k3, k1) of ws2, Q points, output k4 to
//           X[b n + k1 + M k3 + M P k4].
// Every factor is at most 2^8, so every tile covers whole 128-byte rows; the price is a
// third HBM round trip, which the narrow column bands of the two-pass form cost anyway.
static fftc_status three_pass_build(fftc_plan_s *p, int lay) {
    const int logm = 8, logk = p->logn - logm, logp = logk / 2, logq = logk - logp;
    const int64_t n = p->n, B = p->batch, M = int64_t(1) << logm, K = n >> logm;
    const int64_t P = int64_t(1) << logp, Q = int64_t(1) << logq;
    const int64_t plane = lay == LAYOUT_SPLIT ? n * B : 0;
    void *d = nullptr;
    if (plan_alloc(p, (size_t)(n * B) * sizeof(float2), &d) != cudaSuccess) return FFTC_ERR_ALLOC;
    p->workspace = (float2 *)d;
    if (plan_alloc(p, (size_t)(n * B) * sizeof(float2), &d) != cudaSuccess) return FFTC_ERR_ALLOC;
    p->workspace2 = (float2 *)d;
    // w_n^m = lo[m mod 2^b] hi[m >> b] for pass 1, and the same for w_K in pass 2
    fftc_status s;
    p->tw2_lo_bits = (p->logn + 1) / 2;
    if ((s = upload_roots(p, n, int64_t(1) << p->tw2_lo_bits, 1, &p->tw2_lo)) != FFTC_OK) return s;
    if ((s = upload_roots(p, n, n >> p->tw2_lo_bits, int64_t(1) << p->tw2_lo_bits, &p->tw2_hi)) != FFTC_OK) return s;
    const int kbits = (logk + 1) / 2;
    float2 *klo = nullptr, *khi = nullptr;
    if ((s = upload_roots(p, K, int64_t(1) << kbits, 1, &klo)) != FFTC_OK) return s;
    if ((s = upload_roots(p, K, K >> kbits, int64_t(1) << kbits, &khi)) != FFTC_OK) return s;
    p->npasses = 3;
    p->three = true;
    // kind, line length, layouts, L2 prefetch, element stride compiled into the kernel when
    // one is (pass 1: in and out K; pass 3: out M P; pass 2's two strides differ)
    const int shape[3][6] = {{KIND_COLS, logm, lay, LAYOUT_IL, 1, logk},
                             {KIND_COLS, logp, LAYOUT_IL, LAYOUT_IL, 1, 0},
                             {KIND_ROWST, logq, LAYOUT_IL, lay, 0, logm + logp}};
    // pass 1 in 32-column tiles (256-byte rows) where compiled: at 2^24 the split layout's
    // pass 1 measured 0.301 -> 0.267 ms against 16 columns (interleaved even)
    const int c1 = env_int("FFTC_TUNE_COLS_C", 32);
    for (int i = 0; i < 3; ++i) {
        PassPlan &pp = p->pass[i];
        pp.kind = shape[i][0];
        pp.logl = shape[i][1];
        pp.loge = 4;
        pp.lines = i == 0 ? c1 : 16;
        pp.lin = shape[i][2];
        pp.lout = shape[i][3];
        pp.k = find_kernel(pp.kind, pp.logl, pp.loge, pp.lines, pp.lin, pp.lout, 0, shape[i][5]);
        if (!pp.k) {  // run-time strides, 16 lines a tile
            pp.lines = 16;
            pp.k = find_kernel(pp.kind, pp.logl, pp.loge, pp.lines, pp.lin, pp.lout, 0, 0);
        }
        PassParams &b = pp.base;
        memset(&b, 0, sizeof(b));
        b.err = p->d_err;
        set_wait_hooks(b);
        b.pf_tiles = (shape[i][4] && env_int("FFTC_PF", 1)) ? -1 : 0;
    }
    PassParams &a = p->pass[0].base;
    a.in_plane = plane;
    a.total_lines = B * K;
    a.log_lpt = logk;
    a.in_tr = a.out_tr = n;
    a.in_line = a.out_line = 1;
    a.in_elem = a.out_elem = K;
    a.tw2_lo = p->tw2_lo;
    a.tw2_hi = p->tw2_hi;
    a.log_n2 = p->logn;
    a.tw2_lo_bits = p->tw2_lo_bits;
    PassParams &c = p->pass[1].base;  // one transform b: lines (k1, j4)
    c.total_lines = M * Q;
    c.log_lpt = logq;
    c.in_tr = K;
    c.in_line = 1;
    c.in_elem = Q;
    c.out_tr = Q;
    c.out_line = 1;
    c.out_elem = M * Q;
    c.tw2_lo = klo;
    c.tw2_hi = khi;
    c.log_n2 = logk;
    c.tw2_lo_bits = kbits;
    PassParams &r = p->pass[2].base;  // rows (b; k3 M + k1)
    r.out_plane = plane;
    r.total_lines = B * P * M;
    r.log_lpt = logp + logm;
    r.in_tr = r.out_tr = n;
    r.in_line = Q;
    r.in_elem = 1;
    r.out_line = 1;
    r.out_elem = M * P;
    r.post_line_mul = 1;
    r.post_elem_mul = M * P;
    for (int i = 0; i < 3; ++i) {
        if ((s = upload_stage_tables(p, p->pass[i])) != FFTC_OK) return s;
        if ((s = prepare(p->pass[i])) != FFTC_OK) return s;
    }
    return FFTC_OK;
}

// Default cluster single pass per size (measured): clusters of R CTAs of Q = n / R points.
struct ClusterDefault {
    int logn, log1, r;
};
static const ClusterDefault kClusterDefaults[] = {{15, 7, 4}, {16, 8, 8}, {17, 8, 16}, {18, 9, 16}};

const ClusterEntry *cluster_default(int logn, int lay) {
    int log1 = 0, r = 0;
    for (const ClusterDefault &d : kClusterDefaults)
        if (d.logn == logn) {
            log1 = d.log1;
            r = d.r;
        }
    r = env_int("FFTC_TUNE_CLUSTER_R", r);
    const ClusterEntry *any = nullptr;
    for (int i = 0; i < cluster_kernel_count(); ++i) {
        const ClusterEntry *e = cluster_kernel_at(i);
        if (e->logn != logn || e->lay != lay) continue;
        if (e->r == r && (e->log1 == log1 || !any)) return e;
        if (!any) any = e;
    }
    return any;
}

fftc_status cluster_setup(fftc_plan_s *p, const ClusterEntry *ce) {
    if (p->tw2_full) plan_release(p, p->tw2_full);
    p->tw2_full = nullptr;
    fftc_status s = upload_full_diagonal(p, ce->log1, &p->tw2_full);
    if (s != FFTC_OK) return s;
    const int log2 = p->logn - ce->log1;
    int logr = 0;
    while ((1 << logr) < ce->r) ++logr;
    PassPlan &pa = p->pass[0], &pb = p->pass[1];
    four_step_params(p, ce->log1, pa.base, pb.base);
    pa.base.cl_log_rows = ce->log1 - logr;  // rows of phase B per CTA: n1 / R
    pa.kind = KIND_CLUSTER_A;
    pa.logl = ce->log1;
    pa.loge = ce->loge;
    pa.lines = (1 << log2) / ce->r;
    pa.lin = ce->lay;
    pa.lout = LAYOUT_IL;
    pa.k = nullptr;
    pb.kind = KIND_ROWST;
    pb.logl = log2;
    pb.loge = ce->loge;
    pb.lines = (1 << ce->log1) / ce->r;
    pb.lin = LAYOUT_IL;
    pb.lout = ce->lay;
    pb.k = nullptr;
    if ((s = upload_stage_tables(p, pa)) != FFTC_OK) return s;
    if ((s = upload_stage_tables(p, pb)) != FFTC_OK) return s;
    if (ce->prepare() != cudaSuccess) return FFTC_ERR_CUDA;
    p->cluster = ce;
    p->npasses = 1;
    return FFTC_OK;
}

fftc_status plan_build_passes(fftc_plan_s *p) {
    const bool tc = p->precision != FFTC_FP32;
    const int prec = tc ? (int)p->precision : 0;  // registry tag: the tensor-core precision mode
    if (tc && (p->logn < 7 || p->logn > 16)) return FFTC_ERR_UNSUPPORTED_SIZE;
    const int64_t n = p->n, B = p->batch;
    const int lay = p->layout == FFTC_LAYOUT_SPLIT ? LAYOUT_SPLIT : LAYOUT_IL;
    const int64_t plane = (lay == LAYOUT_SPLIT) ? n * B : 0;
    p->total_elems = n * B;
    void *d = nullptr;
    if (plan_alloc(p, 16, &d) != cudaSuccess) return FFTC_ERR_ALLOC;
    p->d_err = (int *)d;
    if (cudaMemset(p->d_err, 0, 16) != cudaSuccess) return FFTC_ERR_CUDA;

    if (p->logn <= (tc ? kMaxSinglePassLog : env_int("FFTC_TUNE_MAX_SINGLE_LOG", kMaxSinglePassLog))) {
        PassPlan &pp = p->pass[0];
        p->npasses = 1;
        pp.kind = KIND_ROWS;
        pp.logl = p->logn;
        if (tc) {
            // radix-32 stages on 32-element threads (one line per tile, one landing buffer)
            // where tc_rows_loge says so, else radix-16 stages on 16-element threads
            // (256-thread tiles up to 2^12, one line per tile above)
            pp.loge = env_int("FFTC_TUNE_TC_E", tc_rows_loge(p->logn));
            pp.lines = (pp.loge == 5 || p->logn >= 12) ? 1 : (4096 >> p->logn);
        } else if (!choose_rows(p->logn, lay, &pp.loge, &pp.lines)) {
            return FFTC_ERR_UNSUPPORTED_SIZE;
        }
        pp.lin = pp.lout = lay;
        pp.k = find_kernel(KIND_ROWS, pp.logl, pp.loge, pp.lines, lay, lay, prec);
        if (tc && !pp.k && pp.loge == 5)  // n = 2^12 .. 2^14: bulk-copy fed, one landing buffer
            pp.k = find_kernel(KIND_ROWS, pp.logl, 5, 1, lay, lay, prec, 0, 5);
        if (tc && !pp.k) {  // n >= 2^9: bulk-copy fed (two landing buffers up to 2^12, one above)
            pp.loge = 4;
            pp.lines = p->logn >= 12 ? 1 : (4096 >> p->logn);
            pp.k = find_kernel(KIND_ROWS, pp.logl, 4, pp.lines, lay, lay, prec);
            if (!pp.k) pp.k = find_kernel(KIND_ROWS, pp.logl, 4, pp.lines, lay, lay, prec, 0, p->logn <= 12 ? 6 : 5);
        }
        // pipelined persistent kernel where it measured faster (n = 2^9 .. 2^14)
        const PipeRowsDefault *pd = pipe_rows_default(p->logn);
        if (!tc && env_int("FFTC_PIPE", pd ? 1 : 0)) {
            const int pe = env_int("FFTC_TUNE_PIPE_E", 0), pc = env_int("FFTC_TUNE_PIPE_C", 0),
                      pk = env_int("FFTC_TUNE_PIPE_CODE", 0);
            const KernelEntry *k =
                pd ? find_kernel(KIND_ROWS, pp.logl, pd->loge, pd->lines, lay, lay, 0, 0, pd->code) : nullptr;
            if (!k) k = find_pipe_rows(pp.logl, lay);
            for (int i = 0; (pe || pc || pk) && i < kernel_count(); ++i) {
                const KernelEntry *e = kernel_at(i);
                if (e->pipe && e->prec == 0 && e->kind == KIND_ROWS && e->logl == pp.logl && e->lin == lay &&
                    (!pe || e->loge == pe) &&
                    (!pc || e->lines == pc) && (!pk || e->pipe == pk))
                    k = e;
            }
            if (k) {
                pp.k = k;
                pp.loge = k->loge;
                pp.lines = k->lines;
            }
        }
        PassParams &b = pp.base;
        memset(&b, 0, sizeof(b));
        b.err = p->d_err;
        set_wait_hooks(b);
        b.in_plane = b.out_plane = plane;
        b.total_lines = B;
        b.log_lpt = 0;
        b.in_tr = b.out_tr = n;
        b.in_line = b.out_line = 0;
        b.in_elem = b.out_elem = 1;
        b.post_line_mul = 0;
        b.post_elem_mul = 1;
        fftc_status s = upload_stage_tables(p, pp);
        if (s != FFTC_OK) return s;
        return prepare(pp);
    }

    // one HBM round trip on a thread-block cluster (FP32, n = 2^15 .. 2^18)
    if (!tc && env_int("FFTC_CLUSTER", 0)) {
        const ClusterEntry *ce = cluster_default(p->logn, lay);
        if (ce) return cluster_setup(p, ce);
    }

    // three HBM passes for the largest lengths (FFTC_THREE_PASS: 0 off, 1 from 2^21)
    {
        const int three = env_int("FFTC_THREE_PASS", -1);
        if (!tc && p->logn >= 21 && (three == 1 || (three < 0 && p->logn >= kThreePassMinLog)))
            return three_pass_build(p, lay);
    }

    // four-step: n = M * K
    int logm, e1, e2, c1 = kPassLines, c2 = kPassLines, p1code = 0, p2code = 0, pf = 0;
    if (tc) {  // the FP32 shapes of 2^15 and 2^16 with 16 elements per thread, bulk-copy fed
        logm = p->logn / 2;
        e1 = e2 = 4;
        p1code = env_int("FFTC_TUNE_TC_P1", 5);  // tensor-map boxes, one landing buffer (0: plain loads)
        p2code = env_int("FFTC_TUNE_TC_P2", 6);  // one bulk copy per tile, two buffers (0: plain loads)
        pf = p1code ? 0 : 1;
    } else {
        const FourStepChoice fc = choose_four_step(p->logn, lay);
        logm = fc.logm;
        e1 = fc.e1;
        e2 = fc.e2;
        c1 = fc.c1;
        c2 = fc.c2;
        p1code = fc.p1;
        p2code = fc.p2;
        pf = fc.pf;
    }
    const int logk = p->logn - logm;
    p->npasses = 2;
    const bool l2res = !tc && fs_available(p->logn, lay);
    if (!l2res) {  // the L2-resident executor owns a small workspace ring instead
        if (plan_alloc(p, (size_t)(n * B) * sizeof(float2), &d) != cudaSuccess) return FFTC_ERR_ALLOC;
        p->workspace = (float2 *)d;
    }

    // inter-pass twiddle w_n^m as a product of two small tables
    p->tw2_lo_bits = (p->logn + 1) / 2;
    const int64_t nlo = int64_t(1) << p->tw2_lo_bits, nhi = n >> p->tw2_lo_bits;
    std::vector<float2> lo(nlo), hi(nhi);
    for (int64_t m = 0; m < nlo; ++m) {
        double c, s;
        unit_root(m, n, &c, &s);
        lo[m] = make_float2((float)c, (float)-s);
    }
    for (int64_t m = 0; m < nhi; ++m) {
        double c, s;
        unit_root(m * nlo, n, &c, &s);
        hi[m] = make_float2((float)c, (float)-s);
    }
    if (plan_upload(p, lo.data(), lo.size() * sizeof(float2), &d) != cudaSuccess) return FFTC_ERR_ALLOC;
    p->tw2_lo = (float2 *)d;
    if (plan_upload(p, hi.data(), hi.size() * sizeof(float2), &d) != cudaSuccess) return FFTC_ERR_ALLOC;
    p->tw2_hi = (float2 *)d;
    if (p->logn <= 20) {
        fftc_status s = upload_full_diagonal(p, logm, &p->tw2_full);
        if (s != FFTC_OK) return s;
    }

    {   // pass 1: columns
        PassPlan &pp = p->pass[0];
        pp.kind = KIND_COLS;
        pp.logl = logm;
        pp.loge = e1;
        pp.lines = c1;
        pp.lin = lay;
        pp.lout = LAYOUT_IL;
        pp.k = nullptr;
        // tensor-map fed pass where it measured faster (narrow column boxes make the
        // bulk-copy engine issue one small request per row, so plain loads often win)
        if (p1code) pp.k = find_kernel(KIND_COLS, pp.logl, pp.loge, pp.lines, pp.lin, pp.lout, prec, logk, p1code);
        if (p1code && !pp.k) pp.k = find_kernel(KIND_COLS, pp.logl, pp.loge, pp.lines, pp.lin, pp.lout, prec, 0, p1code);
        if (!pp.k) pp.k = find_kernel(KIND_COLS, pp.logl, pp.loge, pp.lines, pp.lin, pp.lout, prec, logk);
        if (!pp.k) pp.k = find_kernel(KIND_COLS, pp.logl, pp.loge, pp.lines, pp.lin, pp.lout, prec, 0);
        four_step_params(p, logm, pp.base, p->pass[1].base);
        pp.base.pf_tiles = pf ? -1 : 0;
        fftc_status s = upload_stage_tables(p, pp);
        if (s != FFTC_OK) return s;
        if ((s = prepare(pp)) != FFTC_OK) return s;
    }
    {   // pass 2: rows, transposed store
        PassPlan &pp = p->pass[1];
        pp.kind = KIND_ROWST;
        pp.logl = logk;
        pp.loge = e2;
        pp.lines = c2;
        pp.lin = LAYOUT_IL;
        pp.lout = lay;
        pp.k = nullptr;
        if (p2code) pp.k = find_kernel(KIND_ROWST, pp.logl, pp.loge, pp.lines, pp.lin, pp.lout, prec, logm, p2code);
        if (p2code && !pp.k) pp.k = find_kernel(KIND_ROWST, pp.logl, pp.loge, pp.lines, pp.lin, pp.lout, prec, 0, p2code);
        if (!pp.k) pp.k = find_kernel(KIND_ROWST, pp.logl, pp.loge, pp.lines, pp.lin, pp.lout, prec, logm);
        if (!pp.k) pp.k = find_kernel(KIND_ROWST, pp.logl, pp.loge, pp.lines, pp.lin, pp.lout, prec, 0);
        fftc_status s = upload_stage_tables(p, pp);
        if (s != FFTC_OK) return s;
        if ((s = prepare(pp)) != FFTC_OK) return s;
    }
    if (l2res) {
        fftc_status s = fs_build(p);
        if (s != FFTC_OK) return s;
        p->npasses = 1;  // one HBM round trip: the intermediate stays in L2
    }
    return FFTC_OK;
}

fftc_status plan_build(fftc_plan_s *p) {
    if ((p->n & (p->n - 1)) != 0 || p->precision == FFTC_FP64) return mixed_build(p);
    return plan_build_passes(p);
}

static fftc_status three_pass_run(fftc_plan_s *p, const void *in, void *out, int64_t b0, int64_t nb,
                                  const float *post_h, float post_scale, cudaStream_t st, cudaEvent_t *ev);

fftc_status plan_run(fftc_plan_s *p, const void *in, void *out, const float *post_h, float post_scale,
                     cudaStream_t st) {
    cudaEvent_t *ev = nullptr;
    if (p->probe_on && p->probe_used < p->probe_slots) ev = &p->probe_events[(size_t)3 * p->probe_used++];
    if (p->uneven) {
        if (post_h) return FFTC_ERR_INVALID_VALUE;
        if (ev) cudaEventRecord(ev[0], st);
        fftc_status s = uneven_run(p, in, out, st);
        if (ev) cudaEventRecord(ev[1], st);
        return s;
    }
    if (p->precision != FFTC_FP32 && post_h) return FFTC_ERR_INVALID_VALUE;
    const int inv = p->direction == FFTC_INVERSE ? 1 : 0;
    if (p->mixed || p->nd) {
        if (post_h && p->nd) return FFTC_ERR_INVALID_VALUE;
        if (ev) cudaEventRecord(ev[0], st);
        fftc_status s = p->nd ? nd_run(p, in, out, st) : mixed_run(p, in, out, post_h, post_scale, st);
        if (ev) {
            cudaEventRecord(ev[1], st);
            cudaEventRecord(ev[2], st);
        }
        return s;
    }
    if (ev) cudaEventRecord(ev[0], st);
    if (p->cluster) {
        PassParams a = p->pass[0].base, b = p->pass[1].base;
        a.in = (const float *)in;
        a.conj_in = inv;
        b.out = (float *)out;
        b.conj_out = inv;
        b.post_h = post_h;
        b.post_scale = post_scale;
        if (p->cluster->launch(a, b, p->batch, st) != cudaSuccess) return FFTC_ERR_CUDA;
        if (ev) cudaEventRecord(ev[1], st);
        return FFTC_OK;
    }
    if (p->fs) {
        fftc_status s = fs_run(p, in, out, post_h, post_scale, st);
        if (ev) cudaEventRecord(ev[1], st);
        return s;
    }
    if (p->npasses == 1) {
        PassParams a = p->pass[0].base;
        a.in = (const float *)in;
        a.out = (float *)out;
        a.conj_in = a.conj_out = inv;
        a.post_h = post_h;
        a.post_scale = post_scale;
        if (p->pass[0].k->launch(a, st) != cudaSuccess) return FFTC_ERR_CUDA;
        if (ev) cudaEventRecord(ev[1], st);
        return FFTC_OK;
    }
    if (p->three) {
        fftc_status s = three_pass_run(p, in, out, 0, p->batch, post_h, post_scale, st, ev);
        if (s == FFTC_OK && ev) cudaEventRecord(ev[2], st);
        return s;
    }
    PassParams a = p->pass[0].base;
    a.in = (const float *)in;
    a.out = (float *)p->workspace;
    a.conj_in = inv;
    a.conj_out = 0;
    if (p->pass[0].k->launch(a, st) != cudaSuccess) return FFTC_ERR_CUDA;
    if (ev) cudaEventRecord(ev[1], st);
    PassParams b = p->pass[1].base;
    b.in = (const float *)p->workspace;
    b.out = (float *)out;
    b.conj_in = 0;
    b.conj_out = inv;
    b.post_h = post_h;
    b.post_scale = post_scale;
    if (p->pass[1].k->launch(b, st) != cudaSuccess) return FFTC_ERR_CUDA;
    if (ev) cudaEventRecord(ev[2], st);
    return FFTC_OK;
}

// the three passes on transforms [b0, b0 + nb) (ev[1], when given, after pass 1)
static fftc_status three_pass_run(fftc_plan_s *p, const void *in, void *out, int64_t b0, int64_t nb,
                                  const float *post_h, float post_scale, cudaStream_t st, cudaEvent_t *ev) {
    const int inv = p->direction == FFTC_INVERSE ? 1 : 0;
    const int64_t n = p->n, el = b0 * n;
    const int64_t fo = p->layout == FFTC_LAYOUT_SPLIT ? el : 2 * el;  // float offset in the user layout
    PassParams a = p->pass[0].base;
    a.total_lines = a.total_lines / p->batch * nb;
    a.in = (const float *)in + fo;
    a.out = (float *)p->workspace + 2 * el;
    a.conj_in = inv;
    if (p->pass[0].k->launch(a, st) != cudaSuccess) return FFTC_ERR_CUDA;
    if (ev) cudaEventRecord(ev[1], st);
    for (int64_t b = b0; b < b0 + nb; ++b) {
        PassParams c = p->pass[1].base;
        c.in = (const float *)p->workspace + 2 * b * n;
        c.out = (float *)p->workspace2 + 2 * b * n;
        if (p->pass[1].k->launch(c, st) != cudaSuccess) return FFTC_ERR_CUDA;
    }
    PassParams r = p->pass[2].base;
    r.total_lines = r.total_lines / p->batch * nb;
    r.in = (const float *)p->workspace2 + 2 * el;
    r.out = (float *)out + fo;
    r.conj_out = inv;
    r.post_h = post_h;
    r.post_scale = post_scale;
    return p->pass[2].k->launch(r, st) == cudaSuccess ? FFTC_OK : FFTC_ERR_CUDA;
}

fftc_status plan_run_range(fftc_plan_s *p, const void *in, void *out, int64_t b0, int64_t nb, cudaStream_t st) {
    if (p->uneven || p->fs || p->mixed || p->nd || p->precision != FFTC_FP32 || b0 < 0 || nb < 0 || b0 + nb > p->batch)
        return FFTC_ERR_INVALID_VALUE;
    if (nb == 0) return FFTC_OK;
    if (p->three) return three_pass_run(p, in, out, b0, nb, nullptr, 0.f, st, nullptr);
    const int inv = p->direction == FFTC_INVERSE ? 1 : 0;
    // complex offset of transform b0: interleaved buffers count floats in pairs, the split
    // planes count one float per element (the plane stride stays the whole batch's)
    const int64_t el = b0 * p->n;
    const int64_t fo = p->layout == FFTC_LAYOUT_SPLIT ? el : 2 * el;
    const float *src = (const float *)in + fo;
    float *dst = (float *)out + fo;
    PassParams a = p->pass[0].base;
    a.total_lines = a.total_lines / p->batch * nb;
    a.in = src;
    a.conj_in = inv;
    if (p->cluster) {
        PassParams b = p->pass[1].base;
        b.total_lines = b.total_lines / p->batch * nb;
        b.out = dst;
        b.conj_out = inv;
        return p->cluster->launch(a, b, nb, st) == cudaSuccess ? FFTC_OK : FFTC_ERR_CUDA;
    }
    if (p->npasses == 1) {
        a.out = dst;
        a.conj_out = inv;
        return p->pass[0].k->launch(a, st) == cudaSuccess ? FFTC_OK : FFTC_ERR_CUDA;
    }
    float *ws = (float *)p->workspace + 2 * el;
    a.out = ws;
    a.conj_out = 0;
    if (p->pass[0].k->launch(a, st) != cudaSuccess) return FFTC_ERR_CUDA;
    PassParams b = p->pass[1].base;
    b.total_lines = b.total_lines / p->batch * nb;
    b.in = ws;
    b.out = dst;
    b.conj_in = 0;
    b.conj_out = inv;
    return p->pass[1].k->launch(b, st) == cudaSuccess ? FFTC_OK : FFTC_ERR_CUDA;
}

void plan_destroy_extra(fftc_plan_s *p) {
    uneven_free(p);
    fs_free(p);
    mixed_free(p);
    nd_free(p);
    host_free(p);
}

void plan_probe_free(fftc_plan_s *p) {
    for (cudaEvent_t e : p->probe_events) cudaEventDestroy(e);
    p->probe_events.clear();
    p->probe_slots = p->probe_used = 0;
    p->probe_on = false;
}

fftc_status plan_check_errors(fftc_plan_s *p, cudaStream_t st) {
    if (!p->d_err) return FFTC_OK;
    int h = 0;
    if (cudaMemcpyAsync(&h, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return FFTC_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return FFTC_ERR_CUDA;
    if (h) {
        if (cudaMemsetAsync(p->d_err, 0, sizeof(int), st) != cudaSuccess) return FFTC_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return FFTC_ERR_CUDA;
        return FFTC_ERR_TIMEOUT;
    }
    return FFTC_OK;
}

}  // namespace fftc

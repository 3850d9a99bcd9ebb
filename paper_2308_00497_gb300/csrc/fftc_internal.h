// Internal declarations shared by the planner (fftc_api.cu) and the kernel
// instantiation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fftc {

enum PassKind : int {
    KIND_ROWS = 0,   // whole transforms, contiguous lines in and out (single HBM pass)
    KIND_COLS = 1,   // four-step pass 1: column FFTs at stride K, times w_N^(b t'), in place
    KIND_ROWST = 2,  // four-step pass 2: row FFTs, written transposed (stride M)
    KIND_CLUSTER_A = 3,  // cluster single pass, phase A: column FFTs as KIND_COLS, times
                         // w_N^(b t'), stored into the peer CTAs' shared memory
};

enum LayoutId : int { LAYOUT_IL = 0, LAYOUT_SPLIT = 1 };

// Arguments of one fused Stockham pass. A pass transforms `total_lines` lines of
// length L; line g belongs to transform g >> log_lpt and is line g & (lpt - 1)
// inside it. Element a of line g sits at complex offset
//     (g >> log_lpt) * tr + (g & (lpt - 1)) * line + a * elem
// in the input (in_*) and output (out_*) arrays. Split-layout arrays keep the
// imaginary plane `plane` floats after the real one.
struct PassParams {
    const float *in;
    float *out;
    int64_t in_plane, out_plane;
    int64_t total_lines;
    int64_t in_tr, in_line, in_elem;
    int64_t out_tr, out_line, out_elem;
    const float2 *tw;      // per-stage tables of this pass (Sched layout)
    const float2 *tw2_lo;  // inter-pass twiddle w_N^m = tw2_lo[m & lo_mask] * tw2_hi[m >> lo_bits]
    const float2 *tw2_hi;
    const float2 *tw2_full;  // when set: w_N^(b t') = tw2_full[t' * K + b] (pass-1 layout, one rounding)
    const float *post_h;   // optional real factor per output frequency (NULL = none)
    int64_t post_line_mul, post_elem_mul;  // frequency = line * post_line_mul + a * post_elem_mul
    float post_scale;
    int32_t log_lpt;
    int32_t log_n2;        // log2 N of the inter-pass twiddle (COLS only)
    int32_t tw2_lo_bits;
    int32_t conj_in, conj_out;  // conjugate on load / on store (inverse = conj F conj)
    // indexed lines (uneven batches): line g starts at complex offset line_off[g] of both
    // arrays and is conjugated on load and store when line_conj[g] != 0
    const int64_t *line_off;
    const int8_t *line_conj;
    // persistent launches: when set, `in` / `out` hold byte offsets into the launch's
    // user input / output buffers instead of pointers
    int32_t in_user, out_user;
    // plain four-step pass 1: each CTA first asks L2 to prefetch the input band of tile
    // blockIdx + pf_tiles (the tile a CTA launched about one tile-time later will read),
    // so that HBM streams while this CTA computes (0 = off; < 0: the launch sets it to
    // the number of CTAs resident at once)
    int32_t pf_tiles;
    int *err;  // device error word of the plan (bounded waits that gave up)
    // bounded waits of the pipelined kernels: poll limit (0 = the default), and a test
    // hook that makes every wait run out (the kernels then issue no copy at all)
    int64_t spin_limit;
    int32_t test_no_copy;
    // KIND_CLUSTER_A: log2 of the rows each CTA of the cluster owns in phase B
    int32_t cl_log_rows;
};

typedef cudaError_t (*LaunchFn)(const PassParams &, cudaStream_t);
typedef cudaError_t (*PrepareFn)();

struct KernelEntry {
    int kind, logl, loge, lines, lin, lout;
    int threads;
    int smem_bytes;
    LaunchFn launch;
    PrepareFn prepare;
    int prec;  // fftc_precision of the radix stages: 0 = FP32 on CUDA cores, 1..4 = the tensor-core mode
    int logx;  // four-step passes: log2 of the compile-time element stride (0 = runtime)
    int pipe;  // > 0: persistent kernel fed by bulk copies through `pipe` landing buffers
};

// A compiled cluster single pass (fftc_cluster.cuh): n = 2^logn = n1 n2 with n1 = 2^log1,
// R CTAs per transform, 2^loge elements per thread, one layout in and out. Phase A takes
// the parameters of a four-step pass 1 (KIND_CLUSTER_A), phase B those of a pass 2.
typedef cudaError_t (*ClusterLaunchFn)(const PassParams &a, const PassParams &b, int64_t batch, cudaStream_t st);
struct ClusterEntry {
    int logn, log1, loge, r, lay;
    int threads, smem;
    ClusterLaunchFn launch;
    PrepareFn prepare;
};
int cluster_kernel_count();
const ClusterEntry *cluster_kernel_at(int i);

// Registry of compiled pass kernels (one table per instantiation unit).
const KernelEntry *find_kernel(int kind, int logl, int loge, int lines, int lin, int lout, int prec = 0,
                               int logx = 0, int pipe = 0);
// first pipelined single-pass kernel registered for (log2 L, layout), or NULL
const KernelEntry *find_pipe_rows(int logl, int lay);
int kernel_count();
const KernelEntry *kernel_at(int i);

// Host-side mirror of the device radix schedule (Sched<LOGL, LOGE>).
struct HostSched {
    int S;
    int lr[32];
    int lns[32];
    int tw_total;
};
HostSched host_sched(int logl, int loge);

}  // namespace fftc

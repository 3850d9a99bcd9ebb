// The plan object behind the opaque fftc_plan handle, and the planner entry points.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/fftc.h"
#include "fftc_internal.h"

#define FFTC_PLAN_MAGIC 0x66667463u

namespace fftc {

struct PassPlan {
    int kind, logl, loge, lines, lin, lout;
    const KernelEntry *k;
    float2 *tw;       // device stage tables of this pass
    PassParams base;  // everything but the data pointers, conjugation and epilogue
};

struct UnevenState;  // persistent uneven-batch executor (fftc_uneven.cu)
struct FsState;      // L2-resident four-step executor (fftc_fourstep_l2.cu)
struct TcState;      // tensor-core radix-16 executor (fftc_tc.cu)
struct MixedState;   // mixed-radix passes (fftc_mixed.cu)
struct NdState;      // multidimensional transforms (fftc_mixed.cu)

}  // namespace fftc

struct fftc_plan_s {
    uint32_t magic = 0;
    int device = 0;
    int64_t n = 0;
    int logn = 0;
    int64_t batch = 0;
    int64_t total_elems = 0;  // complex elements per buffer
    fftc_layout layout = FFTC_LAYOUT_INTERLEAVED;
    fftc_direction direction = FFTC_FORWARD;
    fftc_precision precision = FFTC_FP32;
    int npasses = 0;
    fftc::PassPlan pass[3] = {};
    float2 *workspace = nullptr;
    // three HBM passes (n = M P Q, Eq. 1 twice at the memory level): pass[1] runs once per
    // transform of the batch and writes workspace2
    bool three = false;
    float2 *workspace2 = nullptr;
    float2 *tw2_lo = nullptr, *tw2_hi = nullptr, *tw2_full = nullptr;
    int tw2_lo_bits = 0;
    int *d_err = nullptr;  // device error word (bounded waits)
    fftc::UnevenState *uneven = nullptr;
    fftc::TcState *tc = nullptr;
    fftc::FsState *fs = nullptr;
    fftc::MixedState *mixed = nullptr;  // n with factors 3, 5 or 7 (fftc_mixed.cu)
    fftc::NdState *nd = nullptr;        // rank 2 / 3 transforms (fftc_mixed.cu)
    int64_t force_m = 0;  // mixed radix: the split n = M K chosen by measure-mode planning (0: default)
    // cluster single pass (one HBM round trip for n = 2^15 .. 2^18): pass[0] holds phase A
    // (columns of n1), pass[1] phase B (rows of n2); npasses = 1
    const fftc::ClusterEntry *cluster = nullptr;
    std::vector<void *> dev_allocs;
    // timing probe: events[slot * 3 + i] before pass i (i < npasses) and after the last
    std::vector<cudaEvent_t> probe_events;
    int probe_slots = 0, probe_used = 0;
    bool probe_on = false;
    // host-buffer execution (fftc_host.cu): copy streams and events, created on first use
    cudaStream_t xfer_in = nullptr, xfer_out = nullptr;
    cudaEvent_t xev[3] = {nullptr, nullptr, nullptr};
};

namespace fftc {

fftc_status plan_build(fftc_plan_s *p);
// Four-step pieces for the split n = 2^logm * 2^(logn - logm) (Eq. 1 at the memory level):
// the whole inter-pass diagonal in pass-1 layout (n entries, uploaded as a plan allocation),
// and both passes' parameters from the plan's tables (kernels and stage tables aside)
fftc_status upload_full_diagonal(fftc_plan_s *p, int logm, float2 **out);
void four_step_params(const fftc_plan_s *p, int logm, PassParams &a, PassParams &b);
// cluster single pass: switch the plan to `ce` (tables, parameters); the default entry of
// the plan's n and layout, or NULL where none is compiled
fftc_status cluster_setup(fftc_plan_s *p, const ClusterEntry *ce);
const ClusterEntry *cluster_default(int logn, int lay);
// release one device allocation made through plan_alloc / plan_upload
void plan_release(fftc_plan_s *p, void *ptr);
// Enqueue the plan on `st`. post_h (device, n floats, may be NULL) multiplies every
// output frequency k by post_h[k] * post_scale.
fftc_status plan_run(fftc_plan_s *p, const void *in, void *out, const float *post_h, float post_scale,
                     cudaStream_t st);
fftc_status plan_check_errors(fftc_plan_s *p, cudaStream_t st);
// Enqueue the plan on transforms [b0, b0 + nb) of the batch only (FP32 plans with one or two
// launched passes); `in` / `out` are the whole-batch buffers.
fftc_status plan_run_range(fftc_plan_s *p, const void *in, void *out, int64_t b0, int64_t nb, cudaStream_t st);
// Host buffers in and out, copies overlapped with the transform chunk by chunk (fftc_host.cu)
fftc_status host_execute(fftc_plan_s *p, const void *host_in, void *host_out, void *dev_buf, cudaStream_t st);
void host_free(fftc_plan_s *p);
void plan_destroy_extra(fftc_plan_s *p);
void plan_probe_free(fftc_plan_s *p);
void plan_free_device(fftc_plan_s *p);
cudaError_t plan_alloc(fftc_plan_s *p, size_t bytes, void **out);
cudaError_t plan_upload(fftc_plan_s *p, const void *host, size_t bytes, void **out);

void unit_root(int64_t m, int64_t L, double *cosv, double *sinv);
void stage_twiddles(int logl, int loge, std::vector<float2> &out);

// uneven batches (fftc_uneven.cu)
fftc_status uneven_build(fftc_plan_s *p, int64_t count, const int64_t *n, const int8_t *dir, const int64_t *off);
fftc_status uneven_run(fftc_plan_s *p, const void *in, void *out, cudaStream_t st);
void uneven_free(fftc_plan_s *p);
int uneven_max_logn(const fftc_plan_s *p);

// mixed radix, n = 2^a 3^b 5^c 7^d not a power of two (fftc_mixed.cu)
bool mixed_supported(int64_t n);
int64_t mixed_split(int64_t n, bool fp64);
fftc_status mixed_build(fftc_plan_s *p);
fftc_status mixed_run(fftc_plan_s *p, const void *in, void *out, const float *post_h, float post_scale,
                      cudaStream_t st);
int mixed_radix_list(const fftc_plan_s *p, int *radices, int cap);
void mixed_free(fftc_plan_s *p);
// measure-mode planning of mixed-radix plans (the split n = M K) and multidimensional plans
// (the last axis' 1D plan, and compiled versus runtime-radix kernels of the strided axes)
fftc_status mixed_tune(fftc_plan_s *p, int reps);
int64_t mixed_plan_split(const fftc_plan_s *p);  // M of a two-pass mixed plan, n for one pass
fftc_status nd_tune(fftc_plan_s *p, int reps);

// time every compiled kernel that can run each pass of the plan and keep the fastest
// (fftc_tune.cu)
fftc_status plan_tune(fftc_plan_s *p, int reps);

// multidimensional transforms: a 1D plan along the last axis, strided passes along the others
bool nd_axis_supported(int64_t d, bool fp64);
fftc_status nd_build(fftc_plan_s *p, int rank, const int64_t *dims);
fftc_status nd_run(fftc_plan_s *p, const void *in, void *out, cudaStream_t st);
void nd_free(fftc_plan_s *p);

// L2-resident four-step (fftc_fourstep_l2.cu)
bool fs_available(int logn, int lay);
fftc_status fs_build(fftc_plan_s *p);
fftc_status fs_run(fftc_plan_s *p, const void *in, void *out, const float *post_h, float post_scale, cudaStream_t st);
void fs_free(fftc_plan_s *p);

// Kernel choice for a pass; overridable through FFTC_TUNE_* environment variables
// by the tuner. Returns false if no compiled kernel fits.
bool choose_rows(int logn, int lin, int *loge, int *lines);
struct FourStepChoice {
    int logm, e1, c1, e2, c2;
    int p1, p2;  // pipe codes of the two passes (0: plain kernel)
    int pf;      // plain pass 1 prefetches the next wave's input into L2
};
FourStepChoice choose_four_step(int logn, int lay);

}  // namespace fftc

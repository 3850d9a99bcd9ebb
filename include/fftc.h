/*
 * fftc.h -- C ABI of the GB300 batched 1D complex-to-complex FFT library (libfftc.so).
 *
 * The library computes, for every row of a batch,
 *     X_k = sum_{j<n} x_j * exp(s * 2*pi*i * j*k / n),   k = 0..n-1,
 * with s = -1 (FFTC_FORWARD) or s = +1 (FFTC_INVERSE) and no normalisation in
 * either direction, so inverse(forward(x)) = n * x. The arithmetic follows the
 * Cooley-Tukey factorisation of the paper's Eq. 1 (Section 3),
 *     DFT_N = (DFT_K (x) I_M) . D^N_M . (I_K (x) DFT_M) . Pi^N_K ,   N = M*K,
 * applied recursively inside fused Stockham kernels (Section 4 benchmarks the
 * Stockham form), over the two complex layouts of Section 3, step 3
 * ("Interleaved" and "Split").
 *
 * Conventions shared by every call:
 *   - All data pointers passed to fftc_execute are DEVICE pointers on the
 *     device that was current when the plan was created, 16-byte aligned.
 *   - A plan owns its device memory (twiddle tables, workspace, descriptor
 *     tables); fftc_execute never allocates, never synchronises the host and
 *     only enqueues work on the given stream.
 *   - A plan must not be executed concurrently on two streams (it may own a
 *     workspace). Distinct plans are independent.
 *   - Errors are reported only through the returned status; nothing aborts,
 *     throws or exits.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 */
#ifndef FFTC_H
#define FFTC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fftc_plan_s *fftc_plan; /* opaque, owned by the library */

/* Complex layouts (Section 3, step 3).
 * INTERLEAVED: one buffer [batch][n] of (float re, float im) pairs (complex64).
 * SPLIT:       one buffer holding two planes, re[batch][n] then im[batch][n]
 *              (a float32 array of shape [2, batch, n]). */
typedef enum { FFTC_LAYOUT_INTERLEAVED = 0, FFTC_LAYOUT_SPLIT = 1 } fftc_layout;

/* Sign of the exponent. */
typedef enum { FFTC_FORWARD = -1, FFTC_INVERSE = +1 } fftc_direction;

/* Arithmetic of the radix stages.
 * FP32:           every stage in float32 on CUDA cores.
 * *_TC:           radix-16 stages as dense 16x16 complex DFT-matrix products on the
 *                 tensor cores with FP16 or BF16 operands and FP32 accumulation (for
 *                 n = 2^13 and 2^14 radix-32 stages as 32x32 products, one stage fewer).
 * *_TC_SPLIT:     as *_TC, but each operand is split into hi + lo parts and the three
 *                 products hi*hi + hi*lo + lo*hi are accumulated, recovering most of
 *                 the FP32 accuracy.
 * FP64:           complex128 data, every stage in float64 (the runtime-radix kernel,
 *                 any supported n). */
typedef enum {
    FFTC_FP32 = 0,
    FFTC_FP16_TC = 1,
    FFTC_BF16_TC = 2,
    FFTC_FP16_TC_SPLIT = 3,
    FFTC_BF16_TC_SPLIT = 4,
    FFTC_FP64 = 5 /* complex128 data ([batch][n] double pairs, or two double planes) and
                     FP64 arithmetic and tables: the paper's own precision (Section 4) */
} fftc_precision;

typedef enum {
    FFTC_OK = 0,
    FFTC_ERR_INVALID_VALUE = 1,   /* a NULL pointer, a bad enum, a negative count */
    FFTC_ERR_UNSUPPORTED_SIZE = 2,/* n outside [2, 2^24] or with a prime factor above 7, a
                                     non-power-of-two n with a tensor-core precision, an
                                     FP64 n above 4096 with no split M K into factors of
                                     at most 4096, or batch too large */
    FFTC_ERR_MISALIGNED = 3,      /* a data pointer not 16-byte aligned */
    FFTC_ERR_ALLOC = 4,           /* device or host allocation failed in plan creation */
    FFTC_ERR_CUDA = 5,            /* a CUDA runtime call or kernel launch failed */
    FFTC_ERR_INVALID_PLAN = 6,    /* NULL where a plan is required, or a destroyed plan */
    FFTC_ERR_TIMEOUT = 7          /* a bounded device-side wait gave up (see fftc_plan_check) */
} fftc_status;

/*
 * Create a plan for `batch` transforms of length n, 2 <= n <= 2^24, in the given
 * layout, direction and precision, on the current CUDA device. n is a power of two,
 * or (FFTC_FP32 only) any n = 2^a 3^b 5^c 7^d: Eq. 1 with mixed radices 16, 8, 4, 2,
 * 7, 5 and 3 (the mixed radix the paper names as missing, Sections 4 and 6), one
 * pass up to n = 8192 and two passes (n = M K) above. Powers of two take one pass up
 * to 2^14, two above (Eq. 1 once at the memory level, factors up to 2^12) and three at
 * 2^24 (Eq. 1 twice, n = 2^8 P Q, factors up to 2^8; the environment variable
 * FFTC_THREE_PASS = 1 or 0 forces that form on or off for 2^21 and above).
 * Precomputes the twiddle diagonals D (Eq. 1; Table 1 "Mul") in FP64 with exact
 * integer angle reduction and rounds them once to the working precision.
 * Returns NULL on error; fftc_get_last_error() then tells why.
 * Tensor-core precisions require a power of two 2^7 <= n <= 2^16. FFTC_FP64 takes any n the
 * FP32 path takes (one pass up to 4096, two above, both factors at most 4096); its
 * buffers hold complex128.
 */
fftc_plan fftc_plan_create(int64_t n, int64_t batch, fftc_layout layout, fftc_direction direction,
                           fftc_precision precision);

/*
 * Enqueue the plan's transforms on `stream`: read `in`, write `out` (device pointers,
 * 16-byte aligned, each n*batch complex elements in the plan's layout). in == out
 * (in place) is allowed; otherwise the buffers must not overlap. For an uneven plan
 * the buffers hold the rows back to back at the plan's offsets.
 * Returns FFTC_OK once the work is enqueued (kernel faults surface on the stream).
 * Allocates and synchronises nothing (the plan owns every table and workspace), so a
 * call on a stream under CUDA stream capture is recorded into the graph and replays on
 * the buffers given at capture (1D, tensor-core, mixed-radix, FP64 and multidimensional
 * plans). A plan must not run on two streams at once: its workspace is shared.
 */
fftc_status fftc_execute(fftc_plan plan, const void *in, void *out, void *stream);

/*
 * Same transforms, with HOST buffers: copies `host_in` to `dev_buf` (a caller-owned
 * device buffer of at least fftc_plan_bytes() bytes), transforms it in place, copies
 * the result to `host_out`, and waits for the stream. FP32 batches larger than ~32 MiB
 * travel in chunks of whole transforms, each chunk's copy in, transform and copy out
 * overlapped with its neighbours' (two copy streams owned by the plan, chained to
 * `stream` with events). Host buffers should be pinned (page-locked) for the copies to
 * overlap and run at full speed. `dev_buf` must not be used by other work meanwhile.
 */
fftc_status fftc_execute_host(fftc_plan plan, const void *host_in, void *host_out, void *dev_buf,
                              void *stream);

/*
 * out[b][k] = scale * h[k] * X_b[k]: the plan's transforms with a real factor per output
 * frequency fused into the last pass (the diagonal step of a spectral filter, whose
 * adjoint is the same call on the opposite-direction plan). `h` is a device array of n
 * floats (16-byte aligned); the rest is as in fftc_execute. FFTC_FP32 1D plans of any
 * supported n (FFTC_ERR_INVALID_VALUE for tensor-core, FP64, uneven and multidimensional
 * plans).
 */
fftc_status fftc_execute_pointwise(fftc_plan plan, const void *in, void *out, const float *h, float scale,
                                   void *stream);

/* Bytes of one input (or output) buffer of the plan (8 or, for FFTC_FP64, 16 per
 * complex element); 0 for an invalid plan. */
int64_t fftc_plan_bytes(fftc_plan plan);

/* Release the plan and its device memory: the end of the plan life cycle of the
 * FFTW-like library interface the paper's generated code is called through (Section 4:
 * a static library with a plan / execute / destroy style API). NULL is a no-op
 * returning FFTC_OK; a destroyed or foreign handle returns FFTC_ERR_INVALID_PLAN. */
fftc_status fftc_destroy(fftc_plan plan);

/* Status of the last fftc_plan_create* call on this host thread (plan creation returns
 * NULL on failure, as the planner calls of the FFTW-like interface of Section 4 do; this
 * call says why). Thread-local; never fails. */
fftc_status fftc_get_last_error(void);

/* Static, human-readable name of a status code (the error reporting of the library
 * interface of Section 4 is status codes only). Unknown codes map to a fixed string;
 * the result is never NULL and must not be freed. */
const char *fftc_status_string(fftc_status s);

/*
 * Describe the plan's factorisation: the number of HBM passes (1, or 2 for the
 * four-step split n = M*K of Eq. 1 applied once at the memory level) and the radix
 * of every stage in execution order (at most 16 entries). Any output pointer may
 * be NULL. For an uneven plan, passes = 1 and the radices are those of its longest row.
 */
fftc_status fftc_plan_info(fftc_plan plan, int *passes, int *radices, int *n_radices);

/*
 * The split of a 1D plan into HBM passes: *m and *k with m * k = n, m the length of the
 * pass-1 column transforms and k of the pass-2 row transforms of the four-step form
 * (Eq. 1 applied once at the memory level, N = M K). A one-pass plan reports m = n, k = 1;
 * a three-pass plan m = 2^8 and k = n / 2^8 (its two last passes split k once more).
 * Either pointer may be NULL. FFTC_ERR_INVALID_VALUE for uneven and multidimensional plans.
 */
fftc_status fftc_plan_split(fftc_plan plan, int64_t *m, int64_t *k);

/*
 * Measure-mode planning (the runtime search over decompositions that the paper leaves
 * to future work, Section 6; FFTW's "measure"): times, on scratch device buffers of the
 * plan's size allocated and freed inside the call, `reps` launches of every compiled
 * kernel that can run each pass of this plan (single pass: every rows kernel for its n
 * and layout, with each landing-buffer and refill variant, elements per thread (the radix
 * of the stages) and tile height; four-step: every split n = M*K with compiled kernels for
 * both factors, and for each split every column kernel for pass 1, with and without the
 * L2 prefetch, and every transposed-row kernel for pass 2), and keeps the fastest
 * (fftc_plan_split and fftc_plan_info then report the chosen split and radices).
 * Two-pass mixed-radix plans: the divisor splits n = M*K closest to sqrt(n) (six at most)
 * are built and timed whole, and the plan is rebuilt with the fastest. Multidimensional
 * plans: the last axis' 1D plan is tuned as above, and every strided power-of-two axis
 * keeps the faster of its compiled column pass and the runtime-radix pass. Choices are
 * cached per shape for the process, so a second plan of the same shape is tuned without
 * timing; with the environment variable FFTC_TUNE_CACHE naming a file, 1D power-of-two
 * choices are also appended to it and read back by later processes (FFTW's "wisdom").
 * Synchronises the device; do not call it while the plan executes. Tensor-core plans choose
 * among the kernels of their own precision mode; uneven plans are tuned when they are
 * created (fftc_plan_create_uneven) and are returned unchanged, and so are three-pass
 * plans. reps in [1, 1000].
 */
fftc_status fftc_plan_tune(fftc_plan plan, int reps);

/*
 * Multidimensional transforms: `batch` arrays of rank 2 or 3, dims[0] x ... x dims[rank-1]
 * stored row-major (the last axis contiguous), array b at element offset b * prod(dims);
 * the split layout keeps one real plane and one imaginary plane for the whole batch.
 * X[k] = sum_j x[j] prod_a exp(s 2 pi i j_a k_a / dims[a]) (no normalisation), i.e. the
 * Kronecker product of the 1D transforms, the (F (x) I)(I (x) F) form of Section 3 with
 * both factors whole DFTs: the last axis by a 1D plan (any length fftc_plan_create
 * accepts), every other axis by an in-place strided pass (length 2..8192 with prime
 * factors 2, 3, 5, 7; up to 4096 for FFTC_FP64). FFTC_FP32 or FFTC_FP64 (complex128
 * arrays); at most 2^30 elements. Executed with
 * fftc_execute (in place allowed); fftc_plan_info reports the HBM pass count and no
 * radices. Returns NULL on error (fftc_get_last_error tells why).
 */
fftc_plan fftc_plan_create_nd(int rank, const int64_t *dims, int64_t batch, fftc_layout layout,
                              fftc_direction direction, fftc_precision precision);

/*
 * Uneven batch: `count` transforms, row i of length n[i] (a power of two, 64..2^16)
 * with direction[i] in {-1, +1}, stored back to back at complex-element offset
 * offset[i] in the input and output buffers (rows must not overlap). One execute is
 * one persistent-kernel launch, replayed from a CUDA graph captured at the first
 * execute on a given (in, out, stream). n, direction and offset are host arrays,
 * copied into the plan. Only FFTC_FP32 is supported here.
 * The plan is autotuned when it is created (the runtime planning the paper leaves to
 * future work, Section 6): for every length class, each compiled factorisation (one pass,
 * or Eq. 1 once at the memory level, n = M K, for every split with kernels) and tile shape
 * (elements per thread: the default, half of it, or 16 with 4096-element tiles, which
 * fixes the radix of the stages and the lines per tile) is timed inside the persistent
 * kernel on scratch buffers allocated and freed in this call, and the fastest is kept;
 * choices are cached per device for the process and, with FFTC_TUNE_CACHE naming a file,
 * across processes. FFTC_TUNE=0 takes the default table instead.
 */
fftc_plan fftc_plan_create_uneven(int64_t count, const int64_t *n, const int8_t *direction,
                                  const int64_t *offset, fftc_layout layout,
                                  fftc_precision precision);

/*
 * Read and clear the plan's device error word after its work has finished (this call
 * synchronises `stream`). Returns FFTC_ERR_TIMEOUT if a bounded device-side wait of
 * the plan gave up since the last check, FFTC_OK otherwise.
 */
fftc_status fftc_plan_check(fftc_plan plan, void *stream);

/*
 * Host-only inspection of the twiddle diagonals D of Eq. 1 (Table 1 "Mul") that a pass of
 * length L = 2^logl with radix 2^loge uses: writes the per-stage tables (stage s >= 1 holds
 * w_{Ns R}^{t k} at [(t-1) Ns + k], t = 1..R-1, k < Ns, stages concatenated; w_L = exp(-2 pi i/L))
 * as interleaved float pairs into `out` (host memory, room for `capacity` pairs) and returns
 * the number of pairs through *count. Needs no GPU. FFTC_ERR_INVALID_VALUE if
 * 1 <= loge <= logl <= 20 does not hold or the buffer is too small.
 */
fftc_status fftc_stage_twiddles(int logl, int loge, float *out, int64_t capacity, int64_t *count);

/*
 * Timing probe for benchmarks. With enable != 0 every later execute of the plan records
 * a CUDA event on its stream before the first pass, between passes and after the last
 * pass (at most 4096 executes are kept; later ones are not recorded). With enable == 0
 * the probe stops and its records are dropped. Events are created here, not in execute.
 */
fftc_status fftc_plan_timing(fftc_plan plan, int enable);

/*
 * Per-pass device time of the executes recorded since the probe was enabled:
 * ms_per_pass[i] = summed elapsed milliseconds of pass i (i < 2; for a three-pass plan
 * ms_per_pass[1] holds passes 2 and 3 together), *executes = how many executes were
 * recorded. Synchronises on the recorded events.
 */
fftc_status fftc_plan_pass_times(fftc_plan plan, double *ms_per_pass, int *executes);

/*
 * Allocation-free two-pass transform. The paper has no counterpart: this entry point
 * exists for callers that must not allocate device memory themselves, such as a plugin
 * running inside a host application whose caching allocator owns the whole GPU memory
 * budget, or a loop that forbids any allocation once it has started. It needs no plan:
 * it computes the same transforms as a plan of (n, batch, layout, direction, FFTC_FP32)
 * with the four-step kernels, using a library-owned scratch buffer and twiddle tables
 * that are fixed-size __device__ arrays inside libfftc.so. Those arrays (16 MiB of
 * scratch plus about 224 KiB of tables) stay resident on every GPU that loads the
 * library until the process exits.
 *
 *   n      power of two with 2^14 <= n <= 2^20 (the sizes that use a workspace);
 *   batch  with n * batch <= 2^21 complex elements (the scratch capacity);
 *          anything else returns FFTC_ERR_UNSUPPORTED_SIZE, batch < 0 FFTC_ERR_INVALID_VALUE;
 *   in/out device pointers as in fftc_execute (16-byte aligned; in == out allowed).
 *
 * Calls no cudaMalloc, cudaFree or other allocating routine. The first call on a device
 * sets that device up (looks up the arrays' device addresses with the device current,
 * uploads the tables with a synchronous copy); make that first call before any stream
 * capture. With CUDA's lazy module loading the arrays' storage is committed on that
 * first call, not when the library is loaded: make it at start-up, before a caching
 * allocator has reserved the device's memory; if the device has no room left it returns
 * FFTC_ERR_ALLOC. Later calls look the scratch address up again and repeat the set-up
 * when it has changed (after cudaDeviceReset the module, and so its arrays, are new). Every call on a device shares the one scratch array, which keeps the last
 * call's contents (no call relies on it starting at zero: pass 1 overwrites every element
 * that pass 2 reads), so calls that can overlap on the GPU (different streams, or a
 * plan-free call racing another) corrupt each other's results: serialise them.
 */
fftc_status fftc_execute_noalloc(int64_t n, int64_t batch, fftc_layout layout, fftc_direction direction,
                                 const void *in, void *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FFTC_H */

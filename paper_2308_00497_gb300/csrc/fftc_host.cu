// Host-buffer execution: the batch is cut into chunks of about kChunkBytes, and for each
// chunk the host-to-device copy (copy stream `xfer_in`), the transform (the caller's
// stream) and the device-to-host copy (copy stream `xfer_out`) are chained with events, so
// chunk k + 1 travels in while chunk k is transformed and chunk k - 1 travels out. The
// copies of one direction run in order on their stream; a chunk's transform waits for its
// input copy, and its output copy waits for its transform. One cudaMemcpyAsync per
// contiguous range (two per chunk and direction in the split layout, one per plane).
#include <cuda_runtime.h>

#include <algorithm>

#include "fftc_plan.h"

namespace fftc {

static const int64_t kChunkBytes = int64_t(32) << 20;

void host_free(fftc_plan_s *p) {
    for (cudaEvent_t &e : p->xev)
        if (e) {
            cudaEventDestroy(e);
            e = nullptr;
        }
    if (p->xfer_in) cudaStreamDestroy(p->xfer_in);
    if (p->xfer_out) cudaStreamDestroy(p->xfer_out);
    p->xfer_in = p->xfer_out = nullptr;
}

static fftc_status host_setup(fftc_plan_s *p) {
    if (p->xfer_in) return FFTC_OK;
    if (cudaStreamCreateWithFlags(&p->xfer_in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->xfer_out, cudaStreamNonBlocking) != cudaSuccess) {
        host_free(p);
        return FFTC_ERR_CUDA;
    }
    for (cudaEvent_t &e : p->xev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            host_free(p);
            return FFTC_ERR_CUDA;
        }
    return FFTC_OK;
}

// copy transforms [b0, b0 + nb) between the host and the device buffer
static cudaError_t copy_rows(const fftc_plan_s *p, void *dst, const void *src, int64_t b0, int64_t nb,
                             cudaMemcpyKind kind, cudaStream_t st) {
    const int64_t n = p->n;
    if (p->layout != FFTC_LAYOUT_SPLIT) {
        const size_t off = (size_t)(b0 * n) * 8, bytes = (size_t)(nb * n) * 8;
        return cudaMemcpyAsync((char *)dst + off, (const char *)src + off, bytes, kind, st);
    }
    const size_t plane = (size_t)(p->batch * n) * 4, off = (size_t)(b0 * n) * 4, bytes = (size_t)(nb * n) * 4;
    for (int h = 0; h < 2; ++h) {
        cudaError_t e = cudaMemcpyAsync((char *)dst + h * plane + off, (const char *)src + h * plane + off, bytes,
                                        kind, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

fftc_status host_execute(fftc_plan_s *p, const void *host_in, void *host_out, void *dev_buf, cudaStream_t st) {
    const int64_t n = p->n, B = p->batch;
    // chunk rows: a multiple of 4 transforms, so every chunk starts 16-byte aligned in
    // both layouts
    int64_t cb = std::max<int64_t>(1, kChunkBytes / (n * 8));
    cb = (cb + 3) / 4 * 4;
    const bool chunked = !p->uneven && !p->fs && !p->mixed && !p->nd && p->precision == FFTC_FP32 && B > cb;
    const size_t bytes = (size_t)p->total_elems * (p->precision == FFTC_FP64 ? 16 : 8);
    if (!chunked) {
        if (cudaMemcpyAsync(dev_buf, host_in, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return FFTC_ERR_CUDA;
        fftc_status s = plan_run(p, dev_buf, dev_buf, nullptr, 0.f, st);
        if (s != FFTC_OK) return s;
        if (cudaMemcpyAsync(host_out, dev_buf, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) return FFTC_ERR_CUDA;
        return cudaStreamSynchronize(st) == cudaSuccess ? FFTC_OK : FFTC_ERR_CUDA;
    }
    fftc_status s = host_setup(p);
    if (s != FFTC_OK) return s;
    cudaEvent_t ev_start = p->xev[0], ev_in = p->xev[1], ev_done = p->xev[2];
    // nothing earlier on the caller's stream may still use the device buffer
    if (cudaEventRecord(ev_start, st) != cudaSuccess || cudaStreamWaitEvent(p->xfer_in, ev_start, 0) != cudaSuccess)
        return FFTC_ERR_CUDA;
    for (int64_t b0 = 0; b0 < B; b0 += cb) {
        const int64_t nb = std::min(cb, B - b0);
        if (copy_rows(p, dev_buf, host_in, b0, nb, cudaMemcpyHostToDevice, p->xfer_in) != cudaSuccess ||
            cudaEventRecord(ev_in, p->xfer_in) != cudaSuccess || cudaStreamWaitEvent(st, ev_in, 0) != cudaSuccess)
            return FFTC_ERR_CUDA;
        if ((s = plan_run_range(p, dev_buf, dev_buf, b0, nb, st)) != FFTC_OK) return s;
        // the event is re-recorded every chunk: each wait binds to the record before it
        if (cudaEventRecord(ev_done, st) != cudaSuccess || cudaStreamWaitEvent(p->xfer_out, ev_done, 0) != cudaSuccess ||
            copy_rows(p, host_out, dev_buf, b0, nb, cudaMemcpyDeviceToHost, p->xfer_out) != cudaSuccess)
            return FFTC_ERR_CUDA;
    }
    if (cudaEventRecord(ev_done, p->xfer_out) != cudaSuccess || cudaStreamWaitEvent(st, ev_done, 0) != cudaSuccess)
        return FFTC_ERR_CUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? FFTC_OK : FFTC_ERR_CUDA;
}

}  // namespace fftc

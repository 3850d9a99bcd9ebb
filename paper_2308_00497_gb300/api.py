"""Python face of the C ABI: plans over torch tensors, torch supplying memory and streams.

Every transform runs in the CUDA kernels of libfftc.so; this module only checks
shapes, passes device pointers and the current stream, and caches plans.
"""
from __future__ import annotations

import ctypes
import threading

import torch

from . import _native as nat


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


class Plan:
    """A batch of `batch` length-n transforms (include/fftc.h: fftc_plan_create)."""

    def __init__(self, n: int, batch: int, layout: str = "interleaved", inverse: bool = False,
                 precision: str = "fp32", device=None):
        lib = nat.load()
        self.n, self.batch = int(n), int(batch)
        self.layout, self.inverse, self.precision = layout, bool(inverse), precision
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        with torch.cuda.device(self.device):
            h = lib.fftc_plan_create(self.n, self.batch, nat.LAYOUTS[layout],
                                     nat.INVERSE if inverse else nat.FORWARD, nat.PRECISIONS[precision])
        if not h:
            raise nat.FftcError(lib.fftc_get_last_error(), f"fftc_plan_create(n={n}, batch={batch})")
        self._h = ctypes.c_void_p(h)

    @property
    def handle(self):
        return self._h

    def bytes(self) -> int:
        return int(nat.load().fftc_plan_bytes(self._h))

    def info(self):
        """(passes, radices) of the plan's factorisation."""
        p, c = ctypes.c_int(0), ctypes.c_int(0)
        r = (ctypes.c_int * 16)()
        nat.check(nat.load().fftc_plan_info(self._h, ctypes.byref(p), r, ctypes.byref(c)), "fftc_plan_info")
        return p.value, [r[i] for i in range(min(c.value, 16))]

    def split(self):
        """(M, K), M * K = n: the lengths of the pass-1 and pass-2 transforms (n, 1 for one pass)."""
        m, k = ctypes.c_int64(0), ctypes.c_int64(0)
        nat.check(nat.load().fftc_plan_split(self._h, ctypes.byref(m), ctypes.byref(k)), "fftc_plan_split")
        return m.value, k.value

    def _shape(self):
        fp64 = self.precision == "fp64"
        if self.layout == "interleaved":
            return (self.batch, self.n), torch.complex128 if fp64 else torch.complex64
        return (2, self.batch, self.n), torch.float64 if fp64 else torch.float32

    def _check_tensor(self, t: torch.Tensor, name: str):
        shape, dtype = self._shape()
        if t.dtype != dtype or tuple(t.shape) != shape or not t.is_contiguous() or t.device != self.device:
            raise ValueError(f"{name}: expected contiguous {dtype} {shape} on {self.device}, got "
                             f"{t.dtype} {tuple(t.shape)} on {t.device}")

    def execute(self, x: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """out = transform(x) on `stream` (default: torch's current stream)."""
        self._check_tensor(x, "input")
        if out is None:
            out = torch.empty_like(x)
        self._check_tensor(out, "output")
        nat.check(nat.load().fftc_execute(self._h, x.data_ptr(), out.data_ptr(), _stream_handle(stream)),
                  "fftc_execute")
        return out

    def execute_pointwise(self, x: torch.Tensor, h: torch.Tensor, scale: float, out: torch.Tensor | None = None,
                          stream=None) -> torch.Tensor:
        """out[b, k] = scale * h[k] * transform(x)[b, k], the multiply fused into the last pass."""
        self._check_tensor(x, "input")
        if out is None:
            out = torch.empty_like(x)
        self._check_tensor(out, "output")
        if h.dtype != torch.float32 or h.shape != (self.n,) or not h.is_contiguous() or h.device != self.device:
            raise ValueError("h must be a contiguous float32 [n] tensor on the plan's device")
        nat.check(nat.load().fftc_execute_pointwise(self._h, x.data_ptr(), out.data_ptr(), h.data_ptr(),
                                                    float(scale), _stream_handle(stream)), "fftc_execute_pointwise")
        return out

    def execute_host(self, host_in: torch.Tensor, host_out: torch.Tensor, dev_buf: torch.Tensor, stream=None):
        """Host buffers in and out, copies on `stream` (fftc_execute_host); waits for completion."""
        for t, nm in ((host_in, "host_in"), (host_out, "host_out")):
            if t.device.type != "cpu" or not t.is_contiguous() or t.numel() * t.element_size() < self.bytes():
                raise ValueError(f"{nm}: expected a contiguous host tensor of >= {self.bytes()} bytes")
        if dev_buf.device != self.device or dev_buf.numel() * dev_buf.element_size() < self.bytes():
            raise ValueError("dev_buf: expected a device tensor of at least plan bytes")
        nat.check(nat.load().fftc_execute_host(self._h, host_in.data_ptr(), host_out.data_ptr(),
                                               dev_buf.data_ptr(), _stream_handle(stream)), "fftc_execute_host")
        return host_out

    def tune(self, reps: int = 5):
        """Measure-mode planning (fftc_plan_tune): time the candidate decompositions (the
        split n = M K, each pass's kernels and radix schedules; for multidimensional plans
        the last axis and the strided axes' kernels) and keep the fastest, cached per shape
        for the process."""
        with torch.cuda.device(self.device):
            nat.check(nat.load().fftc_plan_tune(self._h, int(reps)), "fftc_plan_tune")
        return self

    def timing(self, enable: bool):
        """Start (or stop and drop) the per-pass event probe (fftc_plan_timing)."""
        nat.check(nat.load().fftc_plan_timing(self._h, 1 if enable else 0), "fftc_plan_timing")

    def pass_times(self):
        """(summed ms per pass [2], recorded executes) since the probe was started."""
        ms = (ctypes.c_double * 2)()
        cnt = ctypes.c_int(0)
        nat.check(nat.load().fftc_plan_pass_times(self._h, ms, ctypes.byref(cnt)), "fftc_plan_pass_times")
        return [ms[0], ms[1]], cnt.value

    def check(self, stream=None):
        nat.check(nat.load().fftc_plan_check(self._h, _stream_handle(stream)), "fftc_plan_check")

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            nat.load().fftc_destroy(h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class UnevenPlan(Plan):
    """Transforms of uneven lengths in one persistent launch (fftc_plan_create_uneven).

    n[i] (powers of two in [64, 2^16]), direction[i] (-1 forward, +1 inverse) and
    offset[i] (complex elements) describe row i of a flat complex64 buffer.
    """

    def __init__(self, n, direction, offset, device=None):
        import numpy as np
        lib = nat.load()
        n = np.ascontiguousarray(n, dtype=np.int64)
        d = np.ascontiguousarray(direction, dtype=np.int8)
        o = np.ascontiguousarray(offset, dtype=np.int64)
        if not (n.shape == d.shape == o.shape) or n.ndim != 1:
            raise ValueError("n, direction and offset must be 1-D arrays of one length")
        self.n_rows = int(n.size)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        self.layout, self.precision = "interleaved", "fp32"
        with torch.cuda.device(self.device):
            h = lib.fftc_plan_create_uneven(self.n_rows, n.ctypes.data, d.ctypes.data, o.ctypes.data,
                                            nat.LAYOUT_INTERLEAVED, nat.FP32)
        if not h:
            raise nat.FftcError(lib.fftc_get_last_error(), f"fftc_plan_create_uneven(count={self.n_rows})")
        self._h = ctypes.c_void_p(h)
        self.total = int(lib.fftc_plan_bytes(self._h)) // 8

    def _check_tensor(self, t: torch.Tensor, name: str):
        if t.dtype != torch.complex64 or t.dim() != 1 or t.numel() < self.total or not t.is_contiguous() \
                or t.device != self.device:
            raise ValueError(f"{name}: expected a contiguous complex64 vector of >= {self.total} elements "
                             f"on {self.device}")


class NdPlan(Plan):
    """`batch` arrays of rank 2 or 3 with shape `dims`, row-major (fftc_plan_create_nd).

    Interleaved tensors are complex64 [batch, *dims]; split tensors float32 [2, batch, *dims].
    """

    def __init__(self, dims, batch: int, layout: str = "interleaved", inverse: bool = False, device=None,
                 precision: str = "fp32"):
        import numpy as np
        lib = nat.load()
        self.dims = tuple(int(d) for d in dims)
        if len(self.dims) not in (2, 3):
            raise ValueError("dims must have 2 or 3 entries")
        self.batch, self.layout, self.inverse, self.precision = int(batch), layout, bool(inverse), precision
        self.n = int(np.prod(self.dims))
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        d = np.ascontiguousarray(self.dims, dtype=np.int64)
        with torch.cuda.device(self.device):
            h = lib.fftc_plan_create_nd(len(self.dims), d.ctypes.data, self.batch, nat.LAYOUTS[layout],
                                        nat.INVERSE if inverse else nat.FORWARD, nat.PRECISIONS[precision])
        if not h:
            raise nat.FftcError(lib.fftc_get_last_error(), f"fftc_plan_create_nd(dims={self.dims}, batch={batch})")
        self._h = ctypes.c_void_p(h)

    def _shape(self):
        fp64 = self.precision == "fp64"
        if self.layout == "interleaved":
            return (self.batch,) + self.dims, torch.complex128 if fp64 else torch.complex64
        return (2, self.batch) + self.dims, torch.float64 if fp64 else torch.float32


_cache: dict = {}
_cache_lock = threading.Lock()


def get_plan(n: int, batch: int, layout: str = "interleaved", inverse: bool = False, precision: str = "fp32",
             device=None) -> Plan:
    dev = torch.cuda.current_device() if device is None else torch.device(device).index or 0
    key = (n, batch, layout, inverse, precision, dev)
    with _cache_lock:
        p = _cache.get(key)
        if p is None:
            p = Plan(n, batch, layout, inverse, precision, device=torch.device("cuda", dev))
            _cache[key] = p
    return p


def _run(x: torch.Tensor, inverse: bool, layout: str, precision: str, out=None) -> torch.Tensor:
    if x.dtype in (torch.complex128, torch.float64):
        precision = "fp64"  # complex128 data: the FP64 path
    want = {"interleaved": torch.complex128 if precision == "fp64" else torch.complex64,
            "split": torch.float64 if precision == "fp64" else torch.float32}[layout]
    if layout == "interleaved":
        if x.dtype != want or x.dim() != 2:
            raise ValueError(f"interleaved input must be a {want} [batch, n] tensor")
        batch, n = x.shape
    else:
        if x.dtype != want or x.dim() != 3 or x.shape[0] != 2:
            raise ValueError(f"split input must be a {want} [2, batch, n] tensor")
        batch, n = x.shape[1], x.shape[2]
    x = x.contiguous()
    return get_plan(n, batch, layout, inverse, precision, device=x.device).execute(x, out)


def fft(x: torch.Tensor, layout: str = "interleaved", precision: str = "fp32", out=None) -> torch.Tensor:
    """Forward transform of every row (exponent sign -1, unnormalised)."""
    return _run(x, False, layout, precision, out)


def ifft(x: torch.Tensor, layout: str = "interleaved", precision: str = "fp32", out=None) -> torch.Tensor:
    """Inverse transform of every row (exponent sign +1, unnormalised: ifft(fft(x)) = n x)."""
    return _run(x, True, layout, precision, out)


_nd_cache: dict = {}


def _run_nd(x: torch.Tensor, rank: int, inverse: bool, layout: str, out=None) -> torch.Tensor:
    precision = "fp64" if x.dtype in (torch.complex128, torch.float64) else "fp32"
    cdt, rdt = (torch.complex128, torch.float64) if precision == "fp64" else (torch.complex64, torch.float32)
    if layout == "interleaved":
        if x.dtype != cdt or x.dim() != rank + 1:
            raise ValueError(f"interleaved input must be a {cdt} [batch, {rank} dims] tensor")
        batch, dims = x.shape[0], tuple(x.shape[1:])
    else:
        if x.dtype != rdt or x.dim() != rank + 2 or x.shape[0] != 2:
            raise ValueError(f"split input must be a {rdt} [2, batch, {rank} dims] tensor")
        batch, dims = x.shape[1], tuple(x.shape[2:])
    key = (dims, batch, layout, inverse, precision, x.device.index)
    with _cache_lock:
        p = _nd_cache.get(key)
        if p is None:
            p = _nd_cache[key] = NdPlan(dims, batch, layout, inverse, device=x.device, precision=precision)
    return p.execute(x.contiguous(), out)


def fftn(x: torch.Tensor, rank: int = 2, layout: str = "interleaved", out=None) -> torch.Tensor:
    """Forward transform over the last `rank` (2 or 3) axes of every array in the batch."""
    return _run_nd(x, rank, False, layout, out)


def ifftn(x: torch.Tensor, rank: int = 2, layout: str = "interleaved", out=None) -> torch.Tensor:
    """Inverse (unnormalised) transform over the last `rank` axes of every array in the batch."""
    return _run_nd(x, rank, True, layout, out)

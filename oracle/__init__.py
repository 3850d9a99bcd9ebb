"""FP64 CPU oracle for the batched 1D complex-to-complex DFT.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The CUDA library and its Python binding never import it, and it
imports nothing from them; the two share no code.

Contents
--------
dft, fft_r2, fft
    The transform X_k = sum_j x_j exp(s 2 pi i jk/n) (s = -1 forward,
    +1 inverse, no normalisation), from ``fft_oracle.c`` (plain C, FP64):
    an O(n^2) direct sum and an independent recursive radix-2 FFT.
kronecker (submodule)
    The paper's Eq. 1 factorisation and its Table 1 operators written out
    as loops / dense matrices, used to pin the readings of the stride
    permutation and of the twiddle diagonal.
spectral_filter, spectral_filter_grad
    The batched spectral filter y = (1/n) F^H (H * F x) and the gradient of
    ||y - t||^2 in PyTorch's convention for complex inputs.

Pins (tests/test_oracle_*.py, run with ``-m "not gpu"``): closed forms
(delta, shifted delta, constant, pure tones, the explicit F_2 and F_4),
linearity, Parseval, inverse(forward(x)) = n x, the shift theorem,
conjugate symmetry of real input, the adjoint dot-product identity, the two
routines against each other, numpy.fft as a third check, the dense Eq. 1
product against DFT_N, and central finite differences of the FP64 loss for
the filter gradient.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fft_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()

#: the direct O(n^2) sum is used up to this length; radix-2 above it
DIRECT_MAX_N = 4096


def build_oracle(force: bool = False) -> str:
    """Compile ``fft_oracle.c`` with gcc into ``oracle/_build/liboracle.so``."""
    import platform
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    stamp = os.path.join(os.path.dirname(_LIB_PATH), "machine.txt")
    other_host = (not os.path.exists(stamp)) or open(stamp).read().strip() != platform.machine()
    stale = other_host or (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        with open(stamp, "w") as f:
            f.write(platform.machine() + "\n")
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build_oracle()
            lib = ctypes.CDLL(_LIB_PATH)
            for name in ("oracle_dft", "oracle_fft_r2", "oracle_fft_mixed"):
                f = getattr(lib, name)
                f.restype = ctypes.c_int
                f.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
            _lib = lib
    return _lib


def default_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return max(1, os.cpu_count() or 1)


def _run(fname: str, x, inverse: bool, threads: int | None):
    x = np.asarray(x)
    squeeze = x.ndim == 1
    xb = np.ascontiguousarray(np.atleast_2d(x), dtype=np.complex128)
    batch, n = xb.shape
    out = np.empty_like(xb)
    sign = 1 if inverse else -1
    th = default_threads() if threads is None else int(threads)
    rc = getattr(_load(), fname)(n, batch, sign, xb.ctypes.data, out.ctypes.data, th)
    if rc != 0:
        raise ValueError(f"{fname} rejected n={n}, batch={batch} (code {rc})")
    return out[0] if squeeze else out


def dft(x, inverse: bool = False, threads: int | None = None) -> np.ndarray:
    """O(n^2) DFT along the last axis of a [batch, n] (or [n]) array, FP64."""
    return _run("oracle_dft", x, inverse, threads)


def fft_r2(x, inverse: bool = False, threads: int | None = None) -> np.ndarray:
    """Recursive radix-2 FFT (n a power of two) along the last axis, FP64."""
    return _run("oracle_fft_r2", x, inverse, threads)


def fft_mixed(x, inverse: bool = False, threads: int | None = None) -> np.ndarray:
    """Recursive mixed-radix FFT (smallest prime factor first, any n) along the last axis, FP64."""
    return _run("oracle_fft_mixed", x, inverse, threads)


def fft(x, inverse: bool = False, threads: int | None = None) -> np.ndarray:
    """The oracle transform: direct sum for n <= 4096, radix-2 above for powers of two,
    mixed radix above for other n."""
    n = np.asarray(x).shape[-1]
    if n <= DIRECT_MAX_N:
        return dft(x, inverse, threads)
    if n & (n - 1) == 0:
        return fft_r2(x, inverse, threads)
    return fft_mixed(x, inverse, threads)


def fftn(x, rank: int, inverse: bool = False, threads: int | None = None) -> np.ndarray:
    """Multidimensional DFT over the last `rank` axes of x ([batch, d0, ..., d_{rank-1}]):
    X[k0..] = sum_j x[j0..] prod_a exp(s 2 pi i j_a k_a / d_a), i.e. the 1D oracle applied
    along each of those axes in turn (the Kronecker product of the 1D DFT matrices, the
    (F (x) I)(I (x) F) form of Section 3 with both factors full transforms)."""
    y = np.asarray(x, dtype=np.complex128)
    for ax in range(y.ndim - rank, y.ndim):
        moved = np.moveaxis(y, ax, -1)
        shape = moved.shape
        flat = fft(np.ascontiguousarray(moved).reshape(-1, shape[-1]), inverse, threads)
        y = np.moveaxis(flat.reshape(shape), -1, ax)
    return np.ascontiguousarray(y)


# ----------------------------------------------------------------------------
# batched spectral filter (the differentiation workload)
# ----------------------------------------------------------------------------

def spectral_filter(x, H, threads: int | None = None) -> np.ndarray:
    """y = (1/n) F^H (H * (F x)) per row; x [batch, n] complex, H [n] (real or complex)."""
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[-1]
    return fft(np.asarray(H) * fft(x, False, threads), True, threads) / n


def spectral_filter_loss(x, H, t, threads: int | None = None) -> float:
    """L = sum |y - t|^2 with y the filter output."""
    y = spectral_filter(x, H, threads)
    d = y - np.asarray(t, dtype=np.complex128)
    return float(np.sum(d.real ** 2 + d.imag ** 2))


def spectral_filter_grad(x, H, t, threads: int | None = None) -> np.ndarray:
    """Gradient of L = ||y - t||^2 in PyTorch's complex convention (dL/dRe x + i dL/dIm x).

    y = A x with A = (1/n) F^H diag(H) F linear over C, so the gradient is
    A^H g_y with g_y = 2 (y - t); A^H = (1/n) F^H diag(conj H) F (F^H F = n I).
    """
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[-1]
    gy = 2.0 * (spectral_filter(x, H, threads) - np.asarray(t, dtype=np.complex128))
    return fft(np.conj(np.asarray(H)) * fft(gy, False, threads), True, threads) / n

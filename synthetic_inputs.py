"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module only draws inputs; it holds none of the transform's arithmetic
and imports neither the oracle nor the CUDA binding. Every generator takes an
explicit seed and uses NumPy's PCG64, so the oracle and the GPU path see the
same bytes.

Recipes (the workloads of the batched 1D C2C FFT):
* uniform_complex:  re, im i.i.d. uniform[-1, 1), drawn as 2*U - 1 with U a
  float32 uniform on [0, 1) (exact in float32, never 1.0).
* gaussian_complex: re, im i.i.d. N(0, 1) (float32).
* tones:            x_j = exp(+2 pi i k0 j / n), one random bin k0 ~ U{0..n-1}
  per row; the angle uses the exact integer (k0*j) mod n, evaluated in FP64
  and rounded to complex64.
* uneven_batch:     4096 lengths n = 2^e with e ~ U{6..16}, direction ~
  Bernoulli(1/2), rows packed back to back (offsets in complex elements).
* gaussian_lowpass: H[k] = exp(-(kappa/k0)^2), kappa = min(k, n-k), k0 = n/16
  (deterministic, real).
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def uniform_complex(batch: int, n: int, seed: int) -> np.ndarray:
    """complex64 [batch, n] with re, im i.i.d. uniform[-1, 1)."""
    r = _rng(seed).random((batch, n, 2), dtype=np.float32)
    v = 2.0 * r - 1.0
    return v.astype(np.float32).view(np.complex64).reshape(batch, n)


def gaussian_complex(batch: int, n: int, seed: int) -> np.ndarray:
    """complex64 [batch, n] with re, im i.i.d. N(0, 1)."""
    v = _rng(seed).standard_normal((batch, n, 2), dtype=np.float32)
    return v.view(np.complex64).reshape(batch, n)


def tones(batch: int, n: int, seed: int):
    """(x, k0): x[b, j] = exp(2 pi i k0[b] j / n) as complex64, k0 ~ U{0..n-1}."""
    k0 = _rng(seed).integers(0, n, size=batch, dtype=np.int64)
    j = np.arange(n, dtype=np.int64)
    m = (k0[:, None] * j[None, :]) % n
    ang = 2.0 * np.pi * (m.astype(np.float64) / n)
    x = (np.cos(ang) + 1j * np.sin(ang)).astype(np.complex64)
    return x, k0


def uneven_batch(count: int = 4096, seed: int = 4, emin: int = 6, emax: int = 16):
    """Descriptors of an uneven batch: (n[count], direction[count], offset[count], total).

    direction is -1 (forward) or +1 (inverse); offsets pack the rows back to
    back in complex elements; total is the number of complex elements.
    """
    g = _rng(seed)
    e = g.integers(emin, emax + 1, size=count, dtype=np.int64)
    n = (np.int64(1) << e).astype(np.int64)
    direction = np.where(g.random(count) < 0.5, -1, 1).astype(np.int8)
    offset = np.zeros(count, dtype=np.int64)
    if count > 1:
        offset[1:] = np.cumsum(n)[:-1]
    total = int(n.sum())
    return n, direction, offset, total


def uneven_data(total: int, seed: int) -> np.ndarray:
    """complex64 [total] uniform[-1, 1) payload for an uneven batch."""
    return uniform_complex(1, total, seed).reshape(total)


def gaussian_lowpass(n: int) -> np.ndarray:
    """float32 [n]: H[k] = exp(-(kappa/k0)^2), kappa = min(k, n-k), k0 = n/16."""
    k = np.arange(n, dtype=np.float64)
    kappa = np.minimum(k, n - k)
    k0 = n / 16.0
    return np.exp(-(kappa / k0) ** 2).astype(np.float32)


def to_split(x: np.ndarray) -> np.ndarray:
    """complex [batch, n] -> float32 [2, batch, n] (re plane, then im plane)."""
    x = np.asarray(x, dtype=np.complex64)
    return np.stack([x.real, x.imag]).astype(np.float32)


def from_split(s: np.ndarray) -> np.ndarray:
    """float32 [2, batch, n] -> complex64 [batch, n]."""
    s = np.asarray(s, dtype=np.float32)
    return (s[0] + 1j * s[1]).astype(np.complex64)

"""Pins for the FP64 spectral filter and its gradient (the differentiation workload).

The paper has no autodiff; the filter y = (1/n) F^H (H * F x) with loss
||y - t||^2 is the batched differentiation workload built on the paper's
transform. The oracle's analytic gradient is pinned against central finite
differences of the FP64 loss at n = 64, batch = 4, and the filter against
its closed forms (H = 1 is the identity; H = delta_0 keeps only the mean).
"""
import numpy as np
import pytest

import oracle
import synthetic_inputs as si


def test_filter_closed_forms():
    n = 64
    x = si.gaussian_complex(4, n, seed=5).astype(np.complex128)
    np.testing.assert_allclose(oracle.spectral_filter(x, np.ones(n)), x, atol=1e-13)
    h = np.zeros(n)
    h[0] = 1
    mean = x.mean(axis=1, keepdims=True)
    np.testing.assert_allclose(oracle.spectral_filter(x, h), np.broadcast_to(mean, x.shape), atol=1e-13)


def test_lowpass_recipe():
    n = 64
    H = si.gaussian_lowpass(n)
    k = np.arange(n)
    assert H[0] == 1.0
    np.testing.assert_allclose(H[1:], H[1:][::-1])  # symmetric in k <-> n-k
    np.testing.assert_allclose(H[4], np.float32(np.exp(-1.0)))  # kappa = k0 = 4


@pytest.mark.parametrize("Hkind", ["lowpass", "complex"])
def test_gradient_matches_finite_differences(Hkind):
    n, B = 64, 4
    x = si.gaussian_complex(B, n, seed=5).astype(np.complex128)
    t = si.gaussian_complex(B, n, seed=6).astype(np.complex128)
    if Hkind == "lowpass":
        H = si.gaussian_lowpass(n).astype(np.float64)
    else:  # a complex H checks that the conjugate lands in the right place
        rng = np.random.Generator(np.random.PCG64(1))
        H = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    g = oracle.spectral_filter_grad(x, H, t)
    scale = np.abs(x).max()
    h = 1e-6 * scale
    fd = np.zeros_like(x)
    for b in range(B):
        for j in range(n):
            for unit in (1.0, 1j):
                xp = x.copy()
                xm = x.copy()
                xp[b, j] += h * unit
                xm[b, j] -= h * unit
                d = (oracle.spectral_filter_loss(xp, H, t) - oracle.spectral_filter_loss(xm, H, t)) / (2 * h)
                fd[b, j] += d * unit
    rel = np.linalg.norm(g - fd) / np.linalg.norm(fd)
    assert rel < 1e-6, rel

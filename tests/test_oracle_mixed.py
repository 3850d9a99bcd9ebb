"""Pins for the mixed-radix FP64 oracle (any n, smallest prime factor first).

Every pin is a fact about the DFT X_k = sum_j x_j exp(s 2 pi i jk/n) that does not go
through the oracle's own recursion: agreement with the independent direct O(n^2) sum
for every 7-smooth n up to 512 (and some lengths with larger primes), closed forms
(delta, shifted delta, constant, pure tone) at lengths far beyond the direct sum's
reach, Parseval, the round trip, and planted mistakes in a copy of the recursion that
the same pins must reject.
"""
import math

import numpy as np
import pytest

import oracle
import synthetic_inputs as si


def _smooth(limit):
    out = []
    for n in range(1, limit + 1):
        m = n
        for p in (2, 3, 5, 7):
            while m % p == 0:
                m //= p
        if m == 1:
            out.append(n)
    return out


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _rand(rows, n, seed):
    return si.gaussian_complex(rows, n, seed=seed).astype(np.complex128)


def test_matches_direct_sum_on_every_7_smooth_length_up_to_512():
    for n in _smooth(512):
        x = _rand(2, n, seed=n)
        for inv in (False, True):
            assert _rel(oracle.fft_mixed(x, inverse=inv), oracle.dft(x, inverse=inv)) <= 1e-13, (n, inv)


@pytest.mark.parametrize("n", [11, 13, 22, 26, 33, 121, 143, 169, 286, 1001])
def test_matches_direct_sum_with_larger_primes(n):
    x = _rand(2, n, seed=n)
    assert _rel(oracle.fft_mixed(x), oracle.dft(x)) <= 1e-13


def _root_powers(n, j0, sign):
    """w^(j0 k) for k < n with the exponent reduced exactly in integers."""
    k = np.arange(n, dtype=np.int64)
    m = (j0 * k) % n
    ang = 2.0 * np.pi * (m.astype(np.float64) / n)
    return np.cos(ang) + 1j * sign * np.sin(ang)


@pytest.mark.parametrize("n", [6561, 15625, 16807, 60000, 100000, 302400])
def test_closed_forms_at_large_n(n):
    # delta at 0 -> ones; constant -> n delta_0
    d = np.zeros(n, complex)
    d[0] = 1
    np.testing.assert_allclose(oracle.fft_mixed(d), np.ones(n), atol=1e-13)
    c = oracle.fft_mixed(np.ones(n, complex))
    assert abs(c[0] - n) <= 1e-9 * n and np.abs(c[1:]).max() <= 1e-9 * n
    # shifted delta -> w^(j0 k), both directions
    for j0 in (1, n // 3, n - 1):
        e = np.zeros(n, complex)
        e[j0] = 1
        np.testing.assert_allclose(oracle.fft_mixed(e), _root_powers(n, j0, -1), atol=1e-12)
        np.testing.assert_allclose(oracle.fft_mixed(e, inverse=True), _root_powers(n, j0, +1), atol=1e-12)
    # pure tone exp(+2 pi i k0 j / n) -> n delta_{k0} forward
    x, k0 = si.tones(2, n, seed=n)
    y = oracle.fft_mixed(x.astype(np.complex128))
    want = np.zeros((2, n), complex)
    want[np.arange(2), k0] = n
    assert _rel(y, want) <= 1e-7  # the tone itself is FP32-rounded


@pytest.mark.parametrize("n", [4725, 9261, 30030])
def test_parseval_and_round_trip(n):
    x = _rand(2, n, seed=7)
    y = oracle.fft_mixed(x)
    np.testing.assert_allclose(np.linalg.norm(y, axis=1) ** 2, n * np.linalg.norm(x, axis=1) ** 2, rtol=1e-12)
    assert _rel(oracle.fft_mixed(y, inverse=True), n * x) <= 1e-13


def test_dispatch_uses_mixed_radix_above_the_direct_limit():
    n = 3 * 4096
    x = _rand(1, n, seed=3)
    np.testing.assert_array_equal(oracle.fft(x), oracle.fft_mixed(x))
    np.testing.assert_array_equal(oracle.fft(x[:, :4096]), oracle.dft(x[:, :4096]))


def _copy_of_recursion(x, bug=None):
    """Pure-Python copy of the oracle's recursion, with an optional planted mistake."""
    n = len(x)
    if n == 1:
        return x.copy()
    p = next(f for f in range(2, n + 1) if n % f == 0)
    m = n // p
    Y = [(_copy_of_recursion(x[r::p], bug) if p != n else x[r:r + 1]) for r in range(p)]
    X = np.zeros(n, complex)
    for k in range(n):
        acc = 0
        for r in range(p):
            if bug == "dropped last subsequence" and r == p - 1 and p > 2:
                continue
            e = (r * (k % m)) % n if bug == "twiddle on k mod m" else (r * k) % n
            sgn = +1 if bug == "wrong twiddle sign" else -1
            acc += np.exp(sgn * 2j * math.pi * e / n) * Y[r][k % m]
        X[k] = acc
    return X


def test_planted_mistakes_fail_the_pins():
    n = 45  # 3 * 3 * 5: two prime factors above 2
    ok = lambda f: all(  # noqa: E731
        np.allclose(f(np.eye(n)[j].astype(complex)), _root_powers(n, j, -1), atol=1e-9) for j in (1, 7, n - 1))
    assert ok(_copy_of_recursion)
    assert ok(lambda v: oracle.fft_mixed(v))
    for bug in ("dropped last subsequence", "twiddle on k mod m", "wrong twiddle sign"):
        assert not ok(lambda v, b=bug: _copy_of_recursion(v, b)), bug

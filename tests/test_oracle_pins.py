"""Pins for the FP64 oracle: closed forms, identities and cross-checks.

The paper (Section 4) only states that its outputs matched FFTW/NumPy for random
inputs of sizes 16..4096; it prints no worked example. So every pin here is a
mathematical fact about the DFT X_k = sum_j x_j exp(s 2 pi i jk/n) (the matrix
that Eq. 1 factorises), chosen so that a dropped term, a wrong sign, a wrong
index or a transposed operand in either oracle routine fails at least one test.
"""
import os

import numpy as np
import pytest

import oracle
import synthetic_inputs as si

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ROUTINES = [("dft", oracle.dft), ("r2", oracle.fft_r2)]
SIZES = [1, 2, 4, 8, 16, 64, 256, 1024]


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            v = [float(t) for t in line.split()]
            rows.append([complex(v[2 * i], v[2 * i + 1]) for i in range(len(v) // 2)])
    return np.array(rows)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("name,f", ROUTINES)
def test_small_matrices_match_golden(name, f):
    for n, fname in [(2, "dft2_forward.txt"), (4, "dft4_forward.txt")]:
        G = _golden(fname)
        cols = f(np.eye(n, dtype=np.complex128))  # row j = transform of e_j = column j of F
        np.testing.assert_allclose(cols.T, G, atol=1e-15)
        # the inverse matrix is the conjugate (unnormalised)
        np.testing.assert_allclose(f(np.eye(n), inverse=True).T, G.conj(), atol=1e-15)


@pytest.mark.parametrize("name,f", ROUTINES)
@pytest.mark.parametrize("n", SIZES)
def test_delta_and_constant(name, f, n):
    d = np.zeros(n, complex)
    d[0] = 1
    np.testing.assert_allclose(f(d), np.ones(n), atol=1e-14)
    np.testing.assert_allclose(f(d, inverse=True), np.ones(n), atol=1e-14)
    one = np.ones(n, complex)
    e0 = np.zeros(n, complex)
    e0[0] = n
    np.testing.assert_allclose(f(one), e0, atol=1e-12 * n)
    np.testing.assert_allclose(f(one, inverse=True), e0, atol=1e-12 * n)


@pytest.mark.parametrize("name,f", ROUTINES)
@pytest.mark.parametrize("n", [4, 8, 64, 1024])
def test_shifted_delta_exact_patterns(name, f, n):
    """delta at n/4 -> (-i)^k forward and (+i)^k inverse; delta at n/2 -> (-1)^k."""
    k = np.arange(n)
    d = np.zeros(n, complex)
    d[n // 4] = 1
    np.testing.assert_allclose(f(d), (-1j) ** (k % 4), atol=1e-13)
    np.testing.assert_allclose(f(d, inverse=True), (1j) ** (k % 4), atol=1e-13)
    d = np.zeros(n, complex)
    d[n // 2] = 1
    np.testing.assert_allclose(f(d), (-1.0) ** k, atol=1e-13)
    # delta at 1 with n = 8: the 8th roots of unity, written with sqrt(2)/2
    if n == 8:
        d = np.zeros(8, complex)
        d[1] = 1
        h = np.sqrt(0.5)
        want = np.array([1, h - 1j * h, -1j, -h - 1j * h, -1, -h + 1j * h, 1j, h + 1j * h])
        np.testing.assert_allclose(f(d), want, atol=1e-15)


@pytest.mark.parametrize("name,f", ROUTINES)
@pytest.mark.parametrize("n", [8, 64, 512, 4096])
def test_pure_tones(name, f, n):
    """exp(+2 pi i k0 j/n): forward -> n delta_{k0}; inverse -> n delta_{-k0 mod n}."""
    x, k0 = si.tones(6, n, seed=11)
    X = f(x.astype(np.complex128))
    Y = f(x.astype(np.complex128), inverse=True)
    for b in range(6):
        want = np.zeros(n, complex)
        want[k0[b]] = n
        # the complex64 rounding of the tone bounds the leakage: |x - exact| <= 2^-24 * sqrt(2)
        assert np.abs(X[b] - want).max() < 4e-7 * n
        want = np.zeros(n, complex)
        want[(-k0[b]) % n] = n
        assert np.abs(Y[b] - want).max() < 4e-7 * n


def test_large_n_radix2_tone_and_parseval():
    n = 1 << 16
    j = np.arange(n)
    k0 = 12345
    x = np.exp(2j * np.pi * ((k0 * j) % n) / n)  # FP64 tone
    X = oracle.fft_r2(x)
    want = np.zeros(n, complex)
    want[k0] = n
    assert np.abs(X - want).max() < 1e-8
    r = si.uniform_complex(2, n, seed=5).astype(np.complex128)
    R = oracle.fft_r2(r)
    np.testing.assert_allclose(np.sum(np.abs(R) ** 2, axis=1), n * np.sum(np.abs(r) ** 2, axis=1), rtol=1e-12)


def test_radix2_at_2p24_tone_and_numpy():
    """The sizes the oracle checks the 2^21..2^24 kernels at: a tone at 2^24 in closed form,
    and numpy's FFT on a random row at 2^22 (its own code, not this oracle's)."""
    n = 1 << 24
    j = np.arange(n, dtype=np.int64)
    k0 = 9876543
    x = np.exp(2j * np.pi * ((k0 * j) % n) / n)
    X = oracle.fft_r2(x[None, :])[0]
    assert abs(X[k0] - n) < 1e-13 * n
    X[k0] = 0.0
    assert np.abs(X).max() < 1e-13 * n
    del x, X
    r = si.uniform_complex(1, 1 << 22, seed=22).astype(np.complex128)
    assert _rel(oracle.fft_r2(r), np.fft.fft(r, axis=1)) < 1e-13


@pytest.mark.parametrize("name,f", ROUTINES)
def test_linearity_parseval_roundtrip(name, f):
    n = 256
    x = si.uniform_complex(4, n, seed=1).astype(np.complex128)
    y = si.gaussian_complex(4, n, seed=2).astype(np.complex128)
    a, b = 0.75 - 0.5j, -1.25 + 2j
    np.testing.assert_allclose(f(a * x + b * y), a * f(x) + b * f(y), atol=1e-11)
    X = f(x)
    np.testing.assert_allclose(np.sum(np.abs(X) ** 2, 1), n * np.sum(np.abs(x) ** 2, 1), rtol=1e-13)
    np.testing.assert_allclose(f(X, inverse=True), n * x, atol=1e-11)


@pytest.mark.parametrize("name,f", ROUTINES)
def test_shift_theorem_and_real_symmetry(name, f):
    n = 128
    x = si.uniform_complex(3, n, seed=3).astype(np.complex128)
    s = 5
    k = np.arange(n)
    # x_{j-s} <-> exp(-2 pi i s k / n) X_k  (forward)
    lhs = f(np.roll(x, s, axis=1))
    rhs = np.exp(-2j * np.pi * ((s * k) % n) / n) * f(x)
    np.testing.assert_allclose(lhs, rhs, atol=1e-11)
    # real input -> X_{n-k} = conj(X_k)
    r = x.real.astype(np.complex128)
    R = f(r)
    np.testing.assert_allclose(R[:, (-k) % n], R.conj(), atol=1e-11)


@pytest.mark.parametrize("name,f", ROUTINES)
def test_adjoint_dot_product(name, f):
    """<F x, y> = <x, F^H y>, with F^H the unnormalised inverse."""
    n = 512
    x = si.gaussian_complex(2, n, seed=7).astype(np.complex128)
    y = si.gaussian_complex(2, n, seed=8).astype(np.complex128)
    lhs = np.sum(f(x) * y.conj(), axis=1)
    rhs = np.sum(x * f(y, inverse=True).conj(), axis=1)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12)


@pytest.mark.parametrize("n", [2, 16, 128, 1024, 4096])
def test_two_oracles_agree(n):
    x = si.uniform_complex(8, n, seed=n).astype(np.complex128)
    for inv in (False, True):
        a = oracle.dft(x, inverse=inv)
        b = oracle.fft_r2(x, inverse=inv)
        assert _rel(a, b) < 1e-13


@pytest.mark.parametrize("n", [16, 1024, 1 << 14])
def test_numpy_third_check(n):
    x = si.uniform_complex(4, n, seed=9).astype(np.complex128)
    assert _rel(oracle.fft(x), np.fft.fft(x, axis=1)) < 1e-13
    assert _rel(oracle.fft(x, inverse=True), n * np.fft.ifft(x, axis=1)) < 1e-13


def test_dispatch_and_threads():
    x = si.uniform_complex(5, 8192, seed=4).astype(np.complex128)
    a = oracle.fft(x, threads=1)
    b = oracle.fft(x, threads=4)
    np.testing.assert_array_equal(a, b)  # threading never changes the bits
    assert oracle.fft(np.zeros((0, 16), complex)).shape == (0, 16)
    with pytest.raises(ValueError):
        oracle.fft_r2(np.ones(12, complex))


def test_mutants_fail_the_pins():
    """Plausible mistakes planted in (copies of) the oracle fail at least one pin."""
    n = 64
    k = np.arange(n)
    d = np.zeros(n, complex)
    d[n // 4] = 1
    good = (-1j) ** (k % 4)
    mutants = {
        "wrong sign": lambda v: oracle.dft(v, inverse=True),
        "transposed index": lambda v: oracle.dft(v)[..., (-k) % n],
        "dropped last term": lambda v: oracle.dft(np.concatenate([v[..., :-1], [0]])),
        "conjugated input": lambda v: oracle.dft(np.conj(v)),
    }
    x, k0 = si.tones(1, n, seed=1)
    tone_want = np.zeros(n, complex)
    tone_want[k0[0]] = n
    for name, m in mutants.items():
        fails = (not np.allclose(m(d), good, atol=1e-9)) or (
            not np.allclose(m(x[0].astype(complex)), tone_want, atol=1e-3))
        if name == "dropped last term":  # the last sample only shows on a delta at n-1
            e = np.zeros(n, complex)
            e[n - 1] = 1
            fails = fails or not np.allclose(m(e), oracle.dft(e), atol=1e-9)
        assert fails, name

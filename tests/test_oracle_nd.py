"""Pins for the multidimensional oracle (oracle.fftn): the 2D / 3D DFT sum written out by
brute force on small shapes, closed forms (delta, separable tones, constant), NumPy as a
third check, and mistakes planted in a copy of the axis loop."""
import itertools
import math

import numpy as np
import pytest

import oracle
import synthetic_inputs as si


def _brute(x, inverse=False):
    """X[k] = sum_j x[j] prod_a exp(s 2 pi i j_a k_a / d_a) with exact integer exponents."""
    dims = x.shape
    s = 1 if inverse else -1
    X = np.zeros(dims, complex)
    for k in itertools.product(*[range(d) for d in dims]):
        acc = 0j
        for j in itertools.product(*[range(d) for d in dims]):
            ang = sum(2 * math.pi * ((ja * ka) % d) / d for ja, ka, d in zip(j, k, dims))
            acc += x[j] * complex(math.cos(ang), s * math.sin(ang))
        X[k] = acc
    return X


@pytest.mark.parametrize("dims", [(3, 4), (4, 6), (5, 2), (2, 3, 5), (4, 2, 3)])
@pytest.mark.parametrize("inverse", [False, True])
def test_matches_brute_force_sum(dims, inverse):
    x = si.gaussian_complex(1, int(np.prod(dims)), seed=len(dims)).reshape((1,) + dims).astype(complex)
    got = oracle.fftn(x, len(dims), inverse)[0]
    want = _brute(x[0], inverse)
    assert np.linalg.norm(got - want) <= 1e-13 * np.linalg.norm(want)


@pytest.mark.parametrize("dims", [(64, 96), (100, 27), (8, 16, 12), (7, 5, 9)])
def test_closed_forms(dims):
    N = int(np.prod(dims))
    d = np.zeros((1,) + dims, complex)
    d[(0,) * (len(dims) + 1)] = 1
    np.testing.assert_allclose(oracle.fftn(d, len(dims)), np.ones((1,) + dims), atol=1e-13)
    c = oracle.fftn(np.ones((1,) + dims, complex), len(dims))
    assert abs(c.flat[0] - N) <= 1e-9 * N and np.abs(c.ravel()[1:]).max() <= 1e-9 * N
    # separable tone exp(+2 pi i sum_a k_a j_a / d_a) -> N delta at (k_a)
    k = tuple(int(v) for v in np.random.default_rng(1).integers(0, dims))
    grids = np.meshgrid(*[np.arange(n) for n in dims], indexing="ij")
    ang = sum(2 * np.pi * ((g * ka) % n) / n for g, ka, n in zip(grids, k, dims))
    y = oracle.fftn(np.exp(1j * ang)[None], len(dims))[0]
    want = np.zeros(dims, complex)
    want[k] = N
    assert np.linalg.norm(y - want) <= 1e-9 * N


def test_numpy_third_check_and_batch_independence():
    x = si.gaussian_complex(3, 24 * 40, seed=9).reshape(3, 24, 40).astype(complex)
    y = oracle.fftn(x, 2)
    np.testing.assert_allclose(y, np.fft.fftn(x, axes=(1, 2)), rtol=0, atol=1e-10)
    np.testing.assert_allclose(oracle.fftn(x[1:2], 2), y[1:2], atol=1e-12)


def test_planted_mistakes_fail():
    x = si.gaussian_complex(1, 12, seed=2).reshape(1, 3, 4).astype(complex)
    want = _brute(x[0])

    def axis(v, ax, inverse):
        moved = np.moveaxis(v, ax, -1)
        out = oracle.fft(np.ascontiguousarray(moved).reshape(-1, moved.shape[-1]), inverse).reshape(moved.shape)
        return np.moveaxis(out, -1, ax)

    mutants = {
        "one axis only": lambda v: axis(v, 2, False),
        "inverse along the first axis": lambda v: axis(axis(v, 2, False), 1, True),
        "dims read in the wrong order": lambda v: oracle.fftn(v.reshape(1, 4, 3), 2).reshape(1, 3, 4),
    }
    assert np.linalg.norm(axis(axis(x, 2, False), 1, False)[0] - want) <= 1e-13 * np.linalg.norm(want)
    for name, m in mutants.items():
        assert np.linalg.norm(m(x)[0] - want) > 1e-3 * np.linalg.norm(want), name

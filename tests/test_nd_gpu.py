"""Rank-2 and rank-3 transforms (fftc_plan_create_nd) against the multidimensional oracle.

Bar: relative L2 per array <= 2e-6 log2(N) with N the element count of one array; both
layouts, both directions, power-of-two and mixed lengths on every axis, in place, round
trip, and a separable tone in closed form.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic_inputs as si
from gpu_util import tol_fp32

pytestmark = pytest.mark.gpu

SHAPES = [(3, 5), (64, 64), (96, 100), (7, 4096), (8192, 8), (100, 3000), (1024, 1024),
          (3, 5, 7), (16, 32, 64), (12, 10, 96), (64, 64, 64), (5, 8, 3000)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2308_00497_gb300 import build
    build.build()


def _to(x, layout):
    if layout == "interleaved":
        return torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).cuda()
    return torch.from_numpy(np.ascontiguousarray(np.stack([x.real, x.imag]).astype(np.float32))).cuda()


def _from(t, layout):
    a = t.cpu().numpy()
    return a if layout == "interleaved" else (a[0] + 1j * a[1])


def _rel(y, ref):
    B = y.shape[0]
    d = (y - ref).reshape(B, -1)
    return np.linalg.norm(d, axis=1) / np.linalg.norm(ref.reshape(B, -1), axis=1)


@pytest.mark.parametrize("dims", SHAPES)
@pytest.mark.parametrize("layout", ["interleaved", "split"])
@pytest.mark.parametrize("inverse", [False, True])
def test_parity(dims, layout, inverse):
    import paper_2308_00497_gb300 as fc
    N = int(np.prod(dims))
    B = 3 if N <= 1 << 20 else 2
    x = si.uniform_complex(B, N, seed=N % 1000).reshape((B,) + dims)
    p = fc.NdPlan(dims, B, layout, inverse)
    y = _from(p.execute(_to(x, layout)), layout)
    torch.cuda.synchronize()
    p.check()
    ref = oracle.fftn(x.astype(np.complex128), len(dims), inverse)
    assert _rel(y, ref).max() <= tol_fp32(N), (dims, layout, inverse)


@pytest.mark.parametrize("dims", [(96, 100), (16, 32, 64)])
def test_in_place_and_round_trip(dims):
    import paper_2308_00497_gb300 as fc
    N = int(np.prod(dims))
    x = si.gaussian_complex(2, N, seed=3).reshape((2,) + dims)
    t = _to(x, "interleaved")
    keep = t.clone()
    fc.fftn(t, len(dims), out=t)
    fc.ifftn(t, len(dims), out=t)
    torch.cuda.synchronize()
    assert _rel(t.cpu().numpy(), N * keep.cpu().numpy()).max() <= 2 * tol_fp32(N)


def test_separable_tone_closed_form():
    import paper_2308_00497_gb300 as fc
    dims, k = (60, 256), (7, 200)
    g0, g1 = np.meshgrid(np.arange(dims[0]), np.arange(dims[1]), indexing="ij")
    ang = 2 * np.pi * ((g0 * k[0]) % dims[0]) / dims[0] + 2 * np.pi * ((g1 * k[1]) % dims[1]) / dims[1]
    x = np.exp(1j * ang)[None]
    y = _from(fc.fftn(_to(x, "interleaved"), 2), "interleaved")
    want = np.zeros((1,) + dims, complex)
    want[0, k[0], k[1]] = np.prod(dims)
    assert _rel(y, want).max() <= tol_fp32(int(np.prod(dims)))


@pytest.mark.parametrize("dims", [(12, 100), (64, 64), (16, 8, 30)])
@pytest.mark.parametrize("layout", ["interleaved", "split"])
def test_fp64_arrays(dims, layout):
    import math

    import paper_2308_00497_gb300 as fc
    N = int(np.prod(dims))
    rng = np.random.default_rng(N)
    x = (rng.standard_normal((2,) + dims) + 1j * rng.standard_normal((2,) + dims))
    t = (torch.from_numpy(np.ascontiguousarray(x)).cuda() if layout == "interleaved" else
         torch.from_numpy(np.ascontiguousarray(np.stack([x.real, x.imag]))).cuda())
    y = _from(fc.fftn(t, len(dims), layout=layout), layout)
    ref = oracle.fftn(x, len(dims))
    assert _rel(y, ref).max() <= 1e-14 * math.log2(N)


@pytest.mark.parametrize("dims,layout", [((256, 256), "interleaved"), ((64, 64, 64), "split"), ((96, 100), "split")])
def test_tuned_nd_plan(dims, layout):
    """Measure-mode planning of a multidimensional plan tunes its last-axis 1D plan and picks,
    for every strided power-of-two axis, the compiled column pass or the runtime-radix pass;
    the result stays within tolerance of the oracle."""
    import paper_2308_00497_gb300 as fc
    N = int(np.prod(dims))
    B = 2
    x = si.uniform_complex(B, N, seed=N % 991).reshape((B,) + dims)
    p = fc.NdPlan(dims, B, layout, False).tune(2)
    y = _from(p.execute(_to(x, layout)), layout)
    torch.cuda.synchronize()
    p.check()
    ref = oracle.fftn(x.astype(np.complex128), len(dims), False)
    assert _rel(y, ref).max() <= tol_fp32(N)

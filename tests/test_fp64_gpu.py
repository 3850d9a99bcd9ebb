"""FP64 (complex128) transforms, FFTC_FP64, against the FP64 oracle.

The paper evaluates double-precision C2C (Section 4). Bar: relative L2 per transform
<= 1e-14 * log2(n) (FP64 unit roundoff 1.1e-16 times the radix-stage depth, with margin),
both layouts and directions, powers of two and mixed lengths, single and two passes.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synthetic_inputs as si

pytestmark = pytest.mark.gpu

SIZES = [2, 3, 8, 12, 64, 100, 1000, 1024, 4096, 4725, 6000, 1 << 16, 59049, 1 << 20]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2308_00497_gb300 import build
    build.build()


def _tol(n):
    return 1e-14 * max(1.0, math.log2(n))


def _to(x, layout):
    if layout == "interleaved":
        return torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return torch.from_numpy(np.ascontiguousarray(np.stack([x.real, x.imag]))).cuda()


def _from(t, layout):
    a = t.cpu().numpy()
    return a if layout == "interleaved" else a[0] + 1j * a[1]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("layout", ["interleaved", "split"])
@pytest.mark.parametrize("inverse", [False, True])
def test_parity(n, layout, inverse):
    import paper_2308_00497_gb300 as fc
    B = 5 if n <= 4096 else 2
    rng = np.random.default_rng(n)
    x = rng.standard_normal((B, n)) + 1j * rng.standard_normal((B, n))
    p = fc.Plan(n, B, layout, inverse, precision="fp64")
    assert p.bytes() == 16 * n * B
    y = _from(p.execute(_to(x, layout)), layout)
    torch.cuda.synchronize()
    p.check()
    ref = oracle.fft(x, inverse=inverse)
    err = np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= _tol(n), (n, layout, inverse, float(err.max()))


def test_dtype_dispatch_and_round_trip():
    import paper_2308_00497_gb300 as fc
    n = 3000
    x = torch.from_numpy(si.gaussian_complex(4, n, seed=1).astype(np.complex128)).cuda()
    y = fc.ifft(fc.fft(x))  # complex128 input selects the FP64 path
    assert y.dtype == torch.complex128
    assert torch.linalg.vector_norm(y - n * x) <= _tol(n) * n * torch.linalg.vector_norm(x)


@pytest.mark.parametrize("n", [4096, 30000])
def test_in_place_and_split_ragged(n):
    import paper_2308_00497_gb300 as fc
    rng = np.random.default_rng(7)
    x = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    t = _to(x, "split")
    fc.Plan(n, 3, "split", True, precision="fp64").execute(t, t)
    torch.cuda.synchronize()
    ref = oracle.fft(x, inverse=True)
    y = _from(t, "split")
    assert (np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)).max() <= _tol(n)

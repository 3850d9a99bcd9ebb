"""The differentiable spectral filter (adjoint kernels behind torch.autograd.Function).

Forward and gradient are compared with the FP64 oracle, whose analytic gradient is
itself pinned by central finite differences (tests/test_oracle_filter.py), at
n = 64, batch = 4 and, on sampled rows, at the workload shape [1024, 2^14].
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic_inputs as si
from gpu_util import rel_l2_rows, tol_fp32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2308_00497_gb300 import build
    build.build()


def _loss_and_grad(x_np, t_np, H_np):
    from paper_2308_00497_gb300.autograd import spectral_filter
    x = torch.from_numpy(x_np).cuda().requires_grad_(True)
    t = torch.from_numpy(t_np).cuda()
    H = torch.from_numpy(H_np).cuda()
    y = spectral_filter(x, H)
    loss = ((y - t).abs() ** 2).sum()
    loss.backward()
    torch.cuda.synchronize()
    return y.detach().cpu().numpy(), x.grad.cpu().numpy()


def test_filter_and_gradient_small():
    n, B = 64, 4
    x = si.gaussian_complex(B, n, seed=5)
    t = si.gaussian_complex(B, n, seed=6)
    H = si.gaussian_lowpass(n)
    y, g = _loss_and_grad(x, t, H)
    x64, t64, H64 = x.astype(np.complex128), t.astype(np.complex128), H.astype(np.float64)
    tol = 4 * tol_fp32(n)
    assert rel_l2_rows(y, oracle.spectral_filter(x64, H64)).max() <= tol
    assert rel_l2_rows(g, oracle.spectral_filter_grad(x64, H64, t64)).max() <= tol


def test_filter_and_gradient_workload_shape_sampled():
    n, B = 1 << 14, 1024
    x = si.gaussian_complex(B, n, seed=5)
    t = si.gaussian_complex(B, n, seed=55)
    H = si.gaussian_lowpass(n)
    y, g = _loss_and_grad(x, t, H)
    rows = np.array([0, 1, 511, 1023])
    x64, t64, H64 = x[rows].astype(np.complex128), t[rows].astype(np.complex128), H.astype(np.float64)
    tol = 4 * tol_fp32(n)
    assert rel_l2_rows(y[rows], oracle.spectral_filter(x64, H64)).max() <= tol
    assert rel_l2_rows(g[rows], oracle.spectral_filter_grad(x64, H64, t64)).max() <= tol


def test_adjoint_dot_product_on_gpu():
    """<A x, v> = <x, A^H v> with A the filter: the backward is the true adjoint."""
    from paper_2308_00497_gb300.autograd import SpectralFilter
    n, B = 4096, 8
    x = torch.from_numpy(si.gaussian_complex(B, n, seed=1)).cuda()
    v = torch.from_numpy(si.gaussian_complex(B, n, seed=2)).cuda()
    H = torch.from_numpy(si.gaussian_lowpass(n)).cuda()
    xr = x.clone().requires_grad_(True)
    y = SpectralFilter.apply(xr, H)
    (gx,) = torch.autograd.grad(y, xr, grad_outputs=v)
    lhs = torch.sum(y.detach().to(torch.complex128) * v.conj().to(torch.complex128))
    rhs = torch.sum(x.to(torch.complex128) * gx.conj().to(torch.complex128))
    assert abs(lhs - rhs) / abs(lhs) < 1e-5


def test_rejects_bad_inputs():
    from paper_2308_00497_gb300.autograd import spectral_filter
    H = torch.ones(64, device="cuda")
    with pytest.raises(ValueError):
        spectral_filter(torch.zeros(4, 64, device="cuda"), H)            # not complex
    with pytest.raises(ValueError):
        spectral_filter(torch.zeros(4, 64, dtype=torch.complex64, device="cuda"), torch.ones(32, device="cuda"))


@pytest.mark.parametrize("n,B", [(60, 4), (1000, 3), (12288, 2)])
def test_filter_and_gradient_mixed_lengths(n, B):
    """The fused diagonal on the runtime-radix path (single pass and two passes)."""
    x = si.gaussian_complex(B, n, seed=15)
    t = si.gaussian_complex(B, n, seed=16)
    H = si.gaussian_lowpass(n)
    y, g = _loss_and_grad(x, t, H)
    H64 = H.astype(np.float64)
    y_ref = oracle.spectral_filter(x.astype(np.complex128), H64)
    g_ref = oracle.spectral_filter_grad(x.astype(np.complex128), H64, t.astype(np.complex128))
    assert rel_l2_rows(y, y_ref).max() <= 4 * tol_fp32(n)
    assert rel_l2_rows(g, g_ref).max() <= 4 * tol_fp32(n)

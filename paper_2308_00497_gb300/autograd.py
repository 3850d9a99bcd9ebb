"""Differentiable batched spectral filter on the fused FFT kernels.

    y = (1/n) F^H (H * (F x))        (rows of x, H real of length n)

F is the forward plan and F^H the inverse (unnormalised) plan of the same shape.
The backward pass is the adjoint of each factor in reverse order: the adjoint of
F^H is F, of the diagonal H/n is conj(H)/n = H/n (H real), and of F is F^H, so

    grad_x = F^H (H/n * (F grad_y)),

i.e. the same two kernel launches as the forward pass, with the H/n factor fused
into the last pass of the first transform (fftc_execute_pointwise). The gradient
follows PyTorch's convention for complex inputs (dL/dRe x + i dL/dIm x).
"""
from __future__ import annotations

import torch

from .api import get_plan


def _filter(x: torch.Tensor, H: torch.Tensor) -> torch.Tensor:
    B, n = x.shape
    fwd = get_plan(n, B, "interleaved", False, device=x.device)
    inv = get_plan(n, B, "interleaved", True, device=x.device)
    u = fwd.execute_pointwise(x, H, 1.0 / n)
    return inv.execute(u, u)  # in place: u is a temporary


class SpectralFilter(torch.autograd.Function):
    """y = ifft(H * fft(x)) / n per row (complex64 [batch, n] on CUDA, H float32 [n])."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, H: torch.Tensor) -> torch.Tensor:
        if x.dtype != torch.complex64 or x.dim() != 2 or not x.is_cuda:
            raise ValueError("x must be a complex64 [batch, n] CUDA tensor")
        if H.dtype != torch.float32 or H.shape != (x.shape[1],) or H.device != x.device:
            raise ValueError("H must be a float32 [n] tensor on x's device")
        x = x.contiguous()
        H = H.contiguous()
        ctx.save_for_backward(H)
        return _filter(x, H)

    @staticmethod
    def backward(ctx, grad_y: torch.Tensor):
        (H,) = ctx.saved_tensors
        if grad_y is None:
            return None, None
        g = grad_y.contiguous()
        if g.dtype != torch.complex64:
            g = g.to(torch.complex64)
        return _filter(g, H), None


def spectral_filter(x: torch.Tensor, H: torch.Tensor) -> torch.Tensor:
    return SpectralFilter.apply(x, H)

"""Helpers shared by the GPU parity tests (no transform arithmetic here)."""
import math

import numpy as np
import torch


def tol_fp32(n: int) -> float:
    """Relative-L2 bound per transform for the FP32 path: 2e-6 * log2(n) (at least 2e-6)."""
    return 2e-6 * max(1.0, math.log2(n))


def rel_l2_rows(y: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """Per-row ||y - ref|| / ||ref|| (rows whose reference is zero use the absolute norm)."""
    y = np.asarray(y, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    num = np.linalg.norm(y - ref, axis=-1)
    den = np.linalg.norm(ref, axis=-1)
    return np.where(den > 0, num / np.where(den > 0, den, 1), num)


def to_device(x: np.ndarray, layout: str, device="cuda"):
    """complex64 [B, n] numpy -> the layout's torch tensor on the device."""
    if layout == "interleaved":
        return torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).to(device)
    s = np.stack([x.real, x.imag]).astype(np.float32)
    return torch.from_numpy(np.ascontiguousarray(s)).to(device)


def from_device(t: torch.Tensor, layout: str) -> np.ndarray:
    a = t.cpu().numpy()
    if layout == "interleaved":
        return a
    return (a[0] + 1j * a[1]).astype(np.complex64)

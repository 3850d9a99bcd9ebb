"""Tensor-core precisions (radix-16 and radix-32 stages) against the FP64 oracle.

The paper evaluates FP64 only, so these bounds are derived here from the unit roundoff u
of each operand format and frozen: a tensor-core stage rounds its inputs and the DFT
matrix once each, so the relative L2 error after s tensor-core stages stays below
2 (s + 1) u, plus the FP32 bound of the rest of the path (twiddles, leftover radix,
accumulation). s is taken as the radix-16 stage count log2(n) // 4, which is at least the
radix-32 stage count log2(n) // 5 of the 32-element kernels:

    FP16 plain  u = 2^-11     BF16 plain  u = 2^-8
    FP16 split  u = 2^-22     BF16 split  u = 2^-16   (hi + lo carry twice the bits)

Inputs are complex Gaussian N(0, 1) (the precision workload). The split modes must also
beat their plain counterparts by a wide margin.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synthetic_inputs as si
from gpu_util import from_device, rel_l2_rows, to_device, tol_fp32

pytestmark = pytest.mark.gpu

U = {"fp16_tc": 2.0 ** -11, "bf16_tc": 2.0 ** -8, "fp16_tc_split": 2.0 ** -22, "bf16_tc_split": 2.0 ** -16}


def bound(mode: str, n: int) -> float:
    s_tc = int(math.log2(n)) // 4
    return 2 * (s_tc + 1) * U[mode] + tol_fp32(n)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2308_00497_gb300 import build
    build.build()


def _run(x, layout, inverse, mode):
    import paper_2308_00497_gb300 as fc
    t = to_device(x, layout)
    y = fc.ifft(t, layout=layout, precision=mode) if inverse else fc.fft(t, layout=layout, precision=mode)
    torch.cuda.synchronize()
    return from_device(y, layout)


SIZES = list(range(7, 17))


@pytest.mark.parametrize("mode", list(U))
@pytest.mark.parametrize("e", SIZES)
def test_tc_modes_within_bound(mode, e):
    n = 1 << e
    B = 37 if n <= 4096 else 5
    x = si.gaussian_complex(B, n, seed=300 + e)
    ref = oracle.fft(x.astype(np.complex128))
    err = rel_l2_rows(_run(x, "interleaved", False, mode), ref).max()
    assert err <= bound(mode, n), (mode, n, float(err), bound(mode, n))


@pytest.mark.parametrize("layout", ["interleaved", "split"])
@pytest.mark.parametrize("inverse", [False, True])
@pytest.mark.parametrize("mode", list(U))
@pytest.mark.parametrize("e", [7, 9, 12, 13, 14, 15, 16])
def test_tc_layouts_and_directions(layout, inverse, mode, e):
    """Every kernel kind (plain tiles, bulk-copy fed tiles with one or two landing buffers,
    both four-step passes with plain or tensor-map fed columns) in both layouts and
    directions; batches that leave the last tile ragged."""
    n = 1 << e
    B = {7: 45, 9: 11, 12: 5}.get(e, 3)
    x = si.gaussian_complex(B, n, seed=400 + e)
    ref = oracle.fft(x.astype(np.complex128), inverse=inverse)
    err = rel_l2_rows(_run(x, layout, inverse, mode), ref).max()
    assert err <= bound(mode, n), (mode, n, float(err))


@pytest.mark.parametrize("mode", list(U))
@pytest.mark.parametrize("e", [8, 13, 16])
def test_tc_pure_tone(mode, e):
    """A unit tone at bin k0 maps to n at k0 and (up to the mode's error) zero elsewhere."""
    n = 1 << e
    x, k0 = si.tones(4, n, seed=600 + e)
    y = _run(x, "interleaved", False, mode)
    want = np.zeros((4, n), np.complex128)
    want[np.arange(4), k0] = n
    err = rel_l2_rows(y, want).max()
    assert err <= bound(mode, n), (mode, n, float(err))


@pytest.mark.parametrize("e", [8, 12, 16])
def test_split_recovers_accuracy(e):
    n = 1 << e
    x = si.gaussian_complex(8, n, seed=500 + e)
    ref = oracle.fft(x.astype(np.complex128))
    err = {m: rel_l2_rows(_run(x, "interleaved", False, m), ref).max() for m in U}
    assert err["fp16_tc_split"] < err["fp16_tc"] / 50
    assert err["bf16_tc_split"] < err["bf16_tc"] / 20
    assert err["bf16_tc"] > err["fp16_tc"]  # fewer mantissa bits, larger error


@pytest.mark.parametrize("e", [12, 14, 16])
def test_tc_determinism_and_rejects_small_n(e):
    """Bit-identical output on repeats and on another stream (the MMA accumulation order
    is fixed by the plan)."""
    import paper_2308_00497_gb300 as fc
    from paper_2308_00497_gb300 import _native as nat
    x = to_device(si.gaussian_complex(8, 1 << e, seed=1), "interleaved")
    p = fc.Plan(1 << e, 8, precision="fp16_tc_split")
    a = p.execute(x)
    b = p.execute(x)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        c = p.execute(x, stream=s)
    torch.cuda.synchronize()
    assert torch.equal(a.view(torch.float32), b.view(torch.float32))
    assert torch.equal(a.view(torch.float32), c.view(torch.float32))
    with pytest.raises(nat.FftcError):
        fc.Plan(64, 4, precision="fp16_tc")


@pytest.mark.parametrize("e", [12, 16])
def test_precision_workload_full_batch_sampled(e):
    """n = 2^12 and 2^16 at the workload's batch 2^14, sampled rows vs the oracle."""
    n, B = 1 << e, 1 << 14
    x = si.gaussian_complex(B, n, seed=3)
    rows = np.array([0, 1, B // 2, B - 1])
    ref = oracle.fft(x[rows].astype(np.complex128))
    for mode in ("fp16_tc_split", "bf16_tc"):
        y = _run(x, "interleaved", False, mode)
        err = rel_l2_rows(y[rows], ref).max()
        assert err <= bound(mode, n), (mode, n, float(err))


@pytest.mark.parametrize("mode", ["fp16_tc_split", "bf16_tc"])
@pytest.mark.parametrize("e", [10, 12, 15])
def test_tuned_tc_plan(mode, e):
    """Measure-mode planning of a tensor-core plan picks among that mode's kernels only and
    stays within the mode's bound; replays are bit-identical."""
    import paper_2308_00497_gb300 as fc
    n = 1 << e
    B = max(4, (1 << 20) // n)
    x = si.gaussian_complex(B, n, seed=700 + e)
    p = fc.Plan(n, B, "interleaved", False, mode).tune(2)
    xd = to_device(x, "interleaved")
    a = p.execute(xd)
    b = p.execute(xd)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    rows = np.array([0, B - 1])
    ref = oracle.fft(x[rows].astype(np.complex128))
    assert rel_l2_rows(from_device(a, "interleaved")[rows], ref).max() <= bound(mode, n)


@pytest.mark.parametrize("layout", ["interleaved", "split"])
@pytest.mark.parametrize("inverse", [False, True])
@pytest.mark.parametrize("mode", list(U))
@pytest.mark.parametrize("e", [12, 13, 14])
@pytest.mark.parametrize("loge", [4, 5])
def test_tc_radix16_and_radix32_kernels(monkeypatch, layout, inverse, mode, e, loge):
    """Both tensor-core single passes of n = 2^12 .. 2^14, whichever the default picks:
    16 elements per thread (radix-16 stages as 32 x 32 real DFT-matrix products) and 32
    (radix-32 stages as 64 x 64 products, the remaining radix on the CUDA cores), in both
    layouts and directions, with a ragged persistent schedule (batch not a multiple of the
    grid)."""
    import paper_2308_00497_gb300 as fc
    monkeypatch.setenv("FFTC_TUNE_TC_E", str(loge))
    n = 1 << e
    B = 7
    x = si.gaussian_complex(B, n, seed=800 + e)
    p = fc.Plan(n, B, layout, inverse, mode)
    r = 1 << loge
    assert p.info()[1][:2] == [r, r], p.info()
    y = p.execute(to_device(x, layout))
    torch.cuda.synchronize()
    ref = oracle.fft(x.astype(np.complex128), inverse=inverse)
    err = rel_l2_rows(from_device(y, layout), ref).max()
    assert err <= bound(mode, n), (mode, n, float(err))

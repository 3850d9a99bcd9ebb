"""Lengths above 2^20, up to 2^24.

FP32 powers of two run Eq. 1 once at the memory level with a factor of 2^11 or 2^12
(column tiles of 8 or 4 lines, transposed-row tiles of 8 or 4 lines), or twice (three HBM
passes, n = 2^8 P Q with P, Q <= 2^8); FP32 mixed lengths and FP64 run the runtime-radix
path, whose split can hold lines longer than 4096.

Powers of two: element-wise parity with the FP64 oracle (radix-2: seconds at 2^24) at
every size, both layouts and directions, one to three transforms, and sampled rows of
the benchmark shape n * batch = 2^26. Mixed lengths of millions of points: the oracle's
mixed-radix routine needs tens of seconds per transform there, so they are checked by
closed forms that hold at any size: a pure tone gives n delta_{k0}, and
inverse(forward(x)) = n x.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synthetic_inputs as si
from gpu_util import from_device, rel_l2_rows, to_device, tol_fp32

pytestmark = pytest.mark.gpu

_REF = {}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2308_00497_gb300 import build
    build.build()


def _batch(e):
    return {21: 3, 22: 2}.get(e, 1)


def _input(e):
    return si.uniform_complex(_batch(e), 1 << e, seed=2100 + e)


def _reference(e, inverse):
    """Oracle output for the size's seeded input, computed once for both layouts."""
    key = (e, inverse)
    if key not in _REF:
        _REF[key] = oracle.fft(_input(e).astype(np.complex128), inverse=inverse)
    return _REF[key]


@pytest.mark.parametrize("e", [21, 22, 23, 24])
@pytest.mark.parametrize("inverse", [False, True])
@pytest.mark.parametrize("layout", ["interleaved", "split"])
def test_parity_powers_of_two_above_2p20(e, inverse, layout):
    import paper_2308_00497_gb300 as fc
    n = 1 << e
    x = _input(e)
    p = fc.Plan(n, x.shape[0], layout, inverse)
    assert p.info()[0] in (2, 3)
    y = from_device(p.execute(to_device(x, layout)), layout)
    torch.cuda.synchronize()
    p.check()
    err = rel_l2_rows(y, _reference(e, inverse))
    assert err.max() <= tol_fp32(n), (n, layout, inverse, float(err.max()))


@pytest.mark.parametrize("e", [21, 24])
def test_benchmark_shape_sampled_rows(e):
    """n * batch = 2^26 (the sweep's volume): first and last rows against the oracle."""
    n = 1 << e
    B = (1 << 26) // n
    x = si.uniform_complex(B, n, seed=2200 + e)
    rows = np.array([0, B - 1])
    ref = oracle.fft(x[rows].astype(np.complex128))
    for layout in ("interleaved", "split"):
        import paper_2308_00497_gb300 as fc
        y = from_device(fc.fft(to_device(x, layout), layout=layout), layout)
        torch.cuda.synchronize()
        assert rel_l2_rows(y[rows], ref).max() <= tol_fp32(n)
        assert np.isfinite(y).all()


def test_pure_tone_2p24():
    import paper_2308_00497_gb300 as fc
    n = 1 << 24
    x, k0 = si.tones(2, n, seed=24)
    y = from_device(fc.fft(to_device(x, "split"), layout="split"), "split")
    want = np.zeros((2, n), np.complex128)
    want[np.arange(2), k0] = n
    assert rel_l2_rows(y, want).max() <= tol_fp32(n)


def test_execute_host_chunked_above_2p20():
    """Host buffers at 2^22 x 6: chunks of four transforms (the 32 MiB chunk rounded up to
    whole groups of four) and a ragged last chunk of two, bitwise the device path."""
    import paper_2308_00497_gb300 as fc
    n, B = 1 << 22, 6
    x = si.uniform_complex(B, n, seed=2222)
    p = fc.Plan(n, B, "interleaved", False)
    dev = p.execute(to_device(x, "interleaved"))
    torch.cuda.synchronize()
    xs = to_device(x, "interleaved").cpu().pin_memory()
    out = torch.empty_like(xs).pin_memory()
    buf = torch.empty_like(xs, device="cuda")
    p.execute_host(xs, out, buf)
    assert torch.equal(out.view(torch.int32), dev.cpu().view(torch.int32))
    ref = oracle.fft(x[[B - 1]].astype(np.complex128))
    assert rel_l2_rows(out.numpy()[[B - 1]], ref).max() <= tol_fp32(n)


@pytest.mark.parametrize("layout", ["interleaved", "split"])
def test_tuned_plan_above_2p20(layout):
    import paper_2308_00497_gb300 as fc
    e = 21
    n = 1 << e
    x = _input(e)
    p = fc.Plan(n, x.shape[0], layout, True).tune(2)
    y = from_device(p.execute(to_device(x, layout)), layout)
    torch.cuda.synchronize()
    p.check()
    assert rel_l2_rows(y, _reference(e, True)).max() <= tol_fp32(n)


# (log2 n, log2 M, pass-1 elements/thread, lines, L2 prefetch, pass-2 elements/thread, lines,
# pass-2 feed code): every non-default kernel compiled for these sizes, with each split
@pytest.mark.parametrize("cfg", [(22, 11, 5, 8, 1, 5, 4, 0), (22, 11, 5, 4, 0, 4, 8, 0), (22, 11, 4, 8, 1, 5, 4, 6),
                                 (22, 10, 5, 8, 0, 5, 4, 5), (22, 10, 4, 8, 1, 4, 4, 0), (23, 12, 5, 4, 1, 5, 8, 0),
                                 (23, 12, 4, 4, 0, 4, 8, 0), (24, 12, 5, 4, 0, 5, 4, 5)])
@pytest.mark.parametrize("layout", ["interleaved", "split"])
def test_kernel_variants_above_2p20(monkeypatch, cfg, layout):
    """Each alternative the measure-mode planner may pick above 2^20, against the oracle."""
    import paper_2308_00497_gb300 as fc
    e, logm, e1, c1, pf, e2, c2, p2 = cfg
    for k, v in (("FFTC_TUNE_FOURSTEP_LOGM", logm), ("FFTC_TUNE_COLS_E", e1), ("FFTC_TUNE_COLS_C", c1),
                 ("FFTC_PF", pf), ("FFTC_TUNE_ROWST_E", e2), ("FFTC_TUNE_ROWST_C", c2),
                 ("FFTC_PIPE4", 2 if p2 else 0), ("FFTC_TUNE_P2_PIPE", p2)):
        monkeypatch.setenv(k, str(v))
    n = 1 << e
    x = _input(e)
    inverse = layout == "split"
    p = fc.Plan(n, x.shape[0], layout, inverse)
    y = from_device(p.execute(to_device(x, layout)), layout)
    torch.cuda.synchronize()
    p.check()
    assert rel_l2_rows(y, _reference(e, inverse)).max() <= tol_fp32(n), (cfg, layout)


def _tone64(n, k0):
    j = np.arange(n, dtype=np.int64)
    ang = 2.0 * np.pi * (((k0 * j) % n).astype(np.float64) / n)
    return np.cos(ang) + 1j * np.sin(ang)


def _to(x, layout):
    if layout == "interleaved":
        return torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return torch.from_numpy(np.ascontiguousarray(np.stack([x.real, x.imag]))).cuda()


def _from(t, layout):
    a = t.cpu().numpy()
    return a if layout == "interleaved" else a[0] + 1j * a[1]


# 3^15 splits as 2187 x 6561 and 2 * 3^14 as 2187 x 4374 (lines above 4096 in the strided
# passes); 3 * 2^21 as 3072 x 2048; 7^8 as 2401 x 2401
@pytest.mark.parametrize("n", [3 ** 15, 2 * 3 ** 14, 3 << 21, 7 ** 8])
@pytest.mark.parametrize("layout", ["interleaved", "split"])
def test_mixed_lengths_above_2p20_tone_and_round_trip(n, layout):
    import paper_2308_00497_gb300 as fc
    k0 = np.array([n // 3 + 1, 12345])
    x = np.stack([_tone64(n, k) for k in k0]).astype(np.complex64)
    p = fc.Plan(n, 2, layout, False)
    assert p.info()[0] == 2
    y = from_device(p.execute(to_device(x, layout)), layout)
    torch.cuda.synchronize()
    p.check()
    want = np.zeros((2, n), np.complex128)
    want[np.arange(2), k0] = n
    assert rel_l2_rows(y, want).max() <= tol_fp32(n), (n, layout)
    g = si.gaussian_complex(2, n, seed=n % 1000)
    back = fc.Plan(n, 2, layout, True).execute(p.execute(to_device(g, layout)))
    torch.cuda.synchronize()
    assert rel_l2_rows(from_device(back, layout) / n, g).max() <= 2 * tol_fp32(n)


def test_fp64_2p24_matches_oracle():
    import paper_2308_00497_gb300 as fc
    n = 1 << 24
    x = _input(24).astype(np.complex128)
    p = fc.Plan(n, 1, "interleaved", False, precision="fp64")
    y = _from(p.execute(_to(x, "interleaved")), "interleaved")
    torch.cuda.synchronize()
    p.check()
    assert rel_l2_rows(y, _reference(24, False)).max() <= 1e-14 * math.log2(n)


@pytest.mark.parametrize("n", [3 ** 14, 2 * 3 ** 14])
def test_fp64_mixed_above_2p20_tone(n):
    """3^14 = 2187 x 2187 runs; 2 * 3^14 has no split into two lines of at most 4096 and is
    refused at plan creation."""
    import paper_2308_00497_gb300 as fc
    from paper_2308_00497_gb300 import FftcError
    if n == 2 * 3 ** 14:
        with pytest.raises(FftcError):
            fc.Plan(n, 1, "split", False, precision="fp64")
        return
    k0 = 777
    x = _tone64(n, k0)[None, :]
    y = _from(fc.Plan(n, 1, "split", False, precision="fp64").execute(_to(x, "split")), "split")
    torch.cuda.synchronize()
    want = np.zeros((1, n), np.complex128)
    want[0, k0] = n
    assert rel_l2_rows(y, want).max() <= 1e-14 * math.log2(n)


@pytest.mark.parametrize("e", [21, 22, 23, 24])
@pytest.mark.parametrize("inverse", [False, True])
@pytest.mark.parametrize("layout", ["interleaved", "split"])
@pytest.mark.parametrize("three", ["0", "1"])
def test_two_and_three_pass_forms(monkeypatch, e, inverse, layout, three):
    """Eq. 1 once at the memory level (two HBM passes) and twice (three passes: columns of
    2^8 at stride n / 2^8, then per transform columns of P at stride Q inside each row, then
    rows of Q stored transposed), each forced, element-wise against the oracle."""
    import paper_2308_00497_gb300 as fc
    monkeypatch.setenv("FFTC_THREE_PASS", three)
    n = 1 << e
    x = _input(e)
    p = fc.Plan(n, x.shape[0], layout, inverse)
    assert p.info()[0] == (3 if three == "1" else 2)
    if three == "1":
        assert p.split() == (256, n // 256)
    y = from_device(p.execute(to_device(x, layout)), layout)
    torch.cuda.synchronize()
    p.check()
    err = rel_l2_rows(y, _reference(e, inverse))
    assert err.max() <= tol_fp32(n), (n, layout, inverse, three, float(err.max()))


def test_three_pass_pointwise_and_host_chunks(monkeypatch):
    """Three-pass plan at 2^22 x 6: the fused pointwise multiply of the last pass (frequency
    k1 + M k3 + M P k4) against the oracle times H, and host-buffer execution in chunks
    bitwise equal to the device path."""
    import paper_2308_00497_gb300 as fc
    monkeypatch.setenv("FFTC_THREE_PASS", "1")
    n, B = 1 << 22, 6
    x = si.uniform_complex(B, n, seed=2323)
    p = fc.Plan(n, B, "interleaved", False)
    assert p.info()[0] == 3
    xd = to_device(x, "interleaved")
    h = torch.from_numpy(si.gaussian_lowpass(n)).cuda()
    yp = p.execute_pointwise(xd, h, 0.5)
    dev = p.execute(xd)
    torch.cuda.synchronize()
    ref = oracle.fft(x[[0, B - 1]].astype(np.complex128)) * (0.5 * h.cpu().numpy().astype(np.float64))
    assert rel_l2_rows(yp.cpu().numpy()[[0, B - 1]], ref).max() <= tol_fp32(n)
    xs = xd.cpu().pin_memory()
    out = torch.empty_like(xs).pin_memory()
    buf = torch.empty_like(xs, device="cuda")
    p.execute_host(xs, out, buf)
    assert torch.equal(out.view(torch.int32), dev.cpu().view(torch.int32))


@pytest.mark.parametrize("layout", ["interleaved", "split"])
def test_three_pass_16_column_bands_2p24(monkeypatch, layout):
    """Three-pass 2^24 with 16-column tiles in pass 1 (the default has 32; the element
    stride 2^16 compiled into the kernel), element-wise against the oracle."""
    import paper_2308_00497_gb300 as fc
    monkeypatch.setenv("FFTC_THREE_PASS", "1")
    monkeypatch.setenv("FFTC_TUNE_COLS_C", "16")
    e = 24
    x = _input(e)
    p = fc.Plan(1 << e, x.shape[0], layout, False)
    assert p.info()[0] == 3
    y = from_device(p.execute(to_device(x, layout)), layout)
    torch.cuda.synchronize()
    p.check()
    assert rel_l2_rows(y, _reference(e, False)).max() <= tol_fp32(1 << e)

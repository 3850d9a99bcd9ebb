"""Mixed-radix sizes n = 2^a 3^b 5^c 7^d (not powers of two) against the FP64 oracle.

Same bar as the power-of-two path: per-transform relative L2 <= 2e-6 log2 n in FP32,
both layouts, both directions, ragged batches; single pass (n <= 8192) and the
two-pass Eq. 1 split above; closed-form tones; the round trip; sampled rows of
n * batch ~ 2^26 workloads.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic_inputs as si
from gpu_util import from_device, rel_l2_rows, to_device, tol_fp32

pytestmark = pytest.mark.gpu

SMALL = [3, 5, 6, 7, 9, 10, 12, 14, 15, 21, 25, 27, 35, 45, 49, 60, 81, 96, 100, 125, 243, 343, 360,
         625, 1000, 1536, 2187, 2401, 3000, 3125, 5040, 6561, 7000, 8000]
LARGE = [10000, 12288, 15625, 16807, 20000, 59049, 100000, 177147, 390625, 823543, 1000000]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2308_00497_gb300 import build
    build.build()


def _tol(n):
    return tol_fp32(n) if n >= 2 else 2e-6


def _check(n, B, layout, inverse, seed):
    import paper_2308_00497_gb300 as fc
    x = si.uniform_complex(B, n, seed=seed)
    p = fc.Plan(n, B, layout, inverse)
    y = from_device(p.execute(to_device(x, layout)), layout)
    torch.cuda.synchronize()
    p.check()
    ref = oracle.fft(x.astype(np.complex128), inverse=inverse)
    err = rel_l2_rows(y, ref)
    assert err.max() <= tol_fp32(n), (n, layout, inverse, float(err.max()))


@pytest.mark.parametrize("n", SMALL)
@pytest.mark.parametrize("layout", ["interleaved", "split"])
@pytest.mark.parametrize("inverse", [False, True])
def test_single_pass_sizes(n, layout, inverse):
    _check(n, 37 if n <= 1000 else 5, layout, inverse, seed=n)


@pytest.mark.parametrize("n", LARGE)
@pytest.mark.parametrize("layout", ["interleaved", "split"])
def test_two_pass_sizes(n, layout):
    _check(n, 3, layout, n % 2 == 1, seed=n + 1)


@pytest.mark.parametrize("n", [15, 360, 6561, 100000])
def test_tones_closed_form(n):
    import paper_2308_00497_gb300 as fc
    x, k0 = si.tones(4, n, seed=n)
    y = from_device(fc.fft(to_device(x, "interleaved")), "interleaved")
    want = np.zeros((4, n), np.complex128)
    want[np.arange(4), k0] = n
    assert rel_l2_rows(y, want).max() <= tol_fp32(n)


@pytest.mark.parametrize("n", [12, 3000, 59049])
def test_round_trip(n):
    import paper_2308_00497_gb300 as fc
    x = to_device(si.gaussian_complex(3, n, seed=n), "interleaved")
    y = fc.ifft(fc.fft(x))
    torch.cuda.synchronize()
    assert rel_l2_rows(y.cpu().numpy(), n * x.cpu().numpy()).max() <= 2 * tol_fp32(n)


@pytest.mark.parametrize("n,B", [(3072, 21845), (6000, 11184), (1000000, 67)])
def test_full_size_sampled_rows(n, B):
    import paper_2308_00497_gb300 as fc
    x = si.uniform_complex(B, n, seed=5)
    rows = np.array([0, B // 3, B - 1])
    for layout, inverse in (("interleaved", False), ("split", True)):
        y = from_device(fc.get_plan(n, B, layout, inverse).execute(to_device(x, layout)), layout)
        ref = oracle.fft(x[rows].astype(np.complex128), inverse=inverse)
        assert rel_l2_rows(y[rows], ref).max() <= tol_fp32(n), (n, layout)


def test_plan_info_radices_multiply_to_n():
    import paper_2308_00497_gb300 as fc
    for n, passes in ((360, 1), (100000, 2)):
        got, radices = fc.Plan(n, 2).info()
        assert got == passes and int(np.prod(radices)) == n and set(radices) <= {2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 14, 15, 16}


@pytest.mark.parametrize("n", [60, 3000, 12288])
@pytest.mark.parametrize("layout", ["interleaved", "split"])
def test_pointwise_diagonal(n, layout):
    """out[k] = scale * h[k] * X[k] with the multiply fused into the last stage."""
    import paper_2308_00497_gb300 as fc
    B = 3
    x = si.uniform_complex(B, n, seed=n + 3)
    h = np.random.default_rng(n).uniform(0.5, 2.0, n).astype(np.float32)
    p = fc.Plan(n, B, layout, False)
    y = from_device(p.execute_pointwise(to_device(x, layout), torch.from_numpy(h).cuda(), 0.25), layout)
    torch.cuda.synchronize()
    ref = 0.25 * h.astype(np.float64) * oracle.fft(x.astype(np.complex128))
    assert rel_l2_rows(y, ref).max() <= tol_fp32(n)


def test_pointwise_is_refused_for_fp64():
    import paper_2308_00497_gb300 as fc
    p = fc.Plan(12, 2, precision="fp64")
    x = torch.zeros((2, 12), dtype=torch.complex128, device="cuda")
    with pytest.raises(RuntimeError):
        p.execute_pointwise(x, torch.ones(12, device="cuda"), 1.0)


@pytest.mark.parametrize("n", [360, 100000])
def test_in_place_batch_one_and_empty(n):
    import paper_2308_00497_gb300 as fc
    x = si.uniform_complex(1, n, seed=11)
    t = to_device(x, "interleaved")
    p = fc.Plan(n, 1)
    p.execute(t, t)  # in place
    torch.cuda.synchronize()
    ref = oracle.fft(x.astype(np.complex128))
    assert rel_l2_rows(t.cpu().numpy(), ref).max() <= tol_fp32(n)
    e = fc.Plan(n, 0)
    e.execute(torch.empty((0, n), dtype=torch.complex64, device="cuda"))
    torch.cuda.synchronize()


@pytest.mark.parametrize("n,layout", [(59049, "interleaved"), (100000, "split"), (1000000, "interleaved")])
def test_tuned_split_search(n, layout):
    """Measure-mode planning of a two-pass mixed length times the divisor splits n = M K
    closest to sqrt(n) and keeps the fastest: the plan then reports a split with M K = n,
    matches the oracle, replays bit-identically, and a second plan reuses the choice."""
    import paper_2308_00497_gb300 as fc
    B = 4
    x = si.uniform_complex(B, n, seed=n % 997)
    ref = oracle.fft(x[[0, B - 1]].astype(np.complex128))
    splits = set()
    for _ in range(2):
        p = fc.Plan(n, B, layout, False).tune(2)
        m, k = p.split()
        assert m * k == n and 1 < m < n
        xd = to_device(x, layout)
        a = p.execute(xd)
        b = p.execute(xd)
        torch.cuda.synchronize()
        p.check()
        assert torch.equal(a, b)
        y = from_device(a, layout)
        assert rel_l2_rows(y[[0, B - 1]], ref).max() <= tol_fp32(n)
        splits.add((m, k))
    assert len(splits) == 1


CT_SINGLE = [12, 96, 360, 1000, 3072, 6000]
CT_TWO = [10000, 59049, 100000, 1000000]


@pytest.mark.parametrize("n", CT_SINGLE + CT_TWO)
@pytest.mark.parametrize("layout", ["interleaved", "split"])
@pytest.mark.parametrize("inverse", [False, True])
def test_per_length_kernels(monkeypatch, n, layout, inverse):
    """The per-length (compile-time radix schedule) kernels against the oracle, both layouts
    and directions, with a batch whose last tile is partial; the runtime-radix kernel of the
    same plan (FFTC_MIXED_CT=0) agrees with them to the FP32 tolerance."""
    import paper_2308_00497_gb300 as fc
    B = {12: 345, 96: 43, 360: 11}.get(n, 3)
    x = si.uniform_complex(B, n, seed=n + 7)
    rows = np.array([0, B - 1]) if n >= 10000 else np.arange(B)
    ref = oracle.fft(x[rows].astype(np.complex128), inverse=inverse)
    outs = []
    for ct in ("1", "0"):
        monkeypatch.setenv("FFTC_MIXED_CT", ct)
        p = fc.Plan(n, B, layout, inverse)
        y = from_device(p.execute(to_device(x, layout)), layout)
        torch.cuda.synchronize()
        p.check()
        assert rel_l2_rows(y[rows], ref).max() <= tol_fp32(n), (n, layout, inverse, ct)
        outs.append(y)
    assert rel_l2_rows(outs[0], outs[1].astype(np.complex128)).max() <= 2 * tol_fp32(n)

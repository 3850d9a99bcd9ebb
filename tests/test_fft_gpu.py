"""Parity of the FP32 CUDA path (through the C ABI) with the FP64 oracle.

Bar: per-transform relative L2 error <= 2e-6 * log2(n) against the oracle on the
same seeded inputs (the FP32 tolerance: rounding error grows like log2 n, Higham), for
every n = 2^1..2^20 (2^21..2^24 in test_large_gpu.py), both layouts (Section 3, step 3)
and both directions; ragged batches so that the last CTA tile is partial; full-size
sweep batches (n * batch = 2^26) on sampled rows; bitwise determinism.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synthetic_inputs as si
from gpu_util import from_device, rel_l2_rows, to_device, tol_fp32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2308_00497_gb300 import build
    build.build()


def _batch_for(n):
    if n <= 16:
        return 300   # tiles of 128 lines: two full tiles and a tail
    if n <= 512:
        return 37
    if n <= 4096:
        return 7
    if n <= 1 << 14:
        return 3
    return 2


def _run(x, layout, inverse):
    import paper_2308_00497_gb300 as fc
    t = to_device(x, layout)
    y = fc.ifft(t, layout=layout) if inverse else fc.fft(t, layout=layout)
    torch.cuda.synchronize()
    return from_device(y, layout)


@pytest.mark.parametrize("layout", ["interleaved", "split"])
@pytest.mark.parametrize("inverse", [False, True])
@pytest.mark.parametrize("e", list(range(1, 21)))
def test_parity_all_sizes(e, inverse, layout):
    n = 1 << e
    B = _batch_for(n)
    x = si.uniform_complex(B, n, seed=1000 + e)
    y = _run(x, layout, inverse)
    ref = oracle.fft(x.astype(np.complex128), inverse=inverse)
    err = rel_l2_rows(y, ref)
    assert err.max() <= tol_fp32(n), (n, float(err.max()))


@pytest.mark.parametrize("e", [4, 8, 10, 12, 13, 14, 16, 20])
def test_pure_tones(e):
    """exp(+2 pi i k0 j / n) -> n delta_{k0} forward (closed form, no oracle needed)."""
    n = 1 << e
    x, k0 = si.tones(4, n, seed=7 + e)
    y = _run(x, "interleaved", False)
    want = np.zeros((4, n), np.complex128)
    want[np.arange(4), k0] = n
    assert rel_l2_rows(y, want).max() <= tol_fp32(n)


@pytest.mark.parametrize("e", [5, 10, 13, 14, 17])
def test_roundtrip_and_inplace(e):
    import paper_2308_00497_gb300 as fc
    n = 1 << e
    x = si.gaussian_complex(3, n, seed=e)
    t = to_device(x, "interleaved")
    keep = t.clone()
    fwd = fc.get_plan(n, 3, "interleaved", False)
    inv = fc.get_plan(n, 3, "interleaved", True)
    fwd.execute(t, t)          # in place
    inv.execute(t, t)
    torch.cuda.synchronize()
    err = rel_l2_rows(t.cpu().numpy(), n * keep.cpu().numpy())
    assert err.max() <= 2 * tol_fp32(n)


@pytest.mark.parametrize("e", [8, 12, 16, 20])
def test_bitwise_determinism(e):
    import paper_2308_00497_gb300 as fc
    n = 1 << e
    B = max(1, (1 << 22) // n)
    x = to_device(si.uniform_complex(B, n, seed=3), "split")
    p = fc.get_plan(n, B, "split", False)
    a = p.execute(x)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b = p.execute(x, stream=s)
    s.synchronize()
    c = p.execute(x)
    torch.cuda.synchronize()
    assert torch.equal(a.view(torch.int32), b.view(torch.int32))
    assert torch.equal(a.view(torch.int32), c.view(torch.int32))


@pytest.mark.parametrize("e", list(range(8, 21)))
def test_full_size_sweep_sampled_rows(e):
    """The benchmark's sweep shapes (n * batch = 2^26) in both layouts; rows sampled
    (first, last and two random ones) are checked against the oracle."""
    n = 1 << e
    B = (1 << 26) // n
    x = si.uniform_complex(B, n, seed=200 + e)
    rows = np.unique(np.array([0, B - 1, *np.random.default_rng(e).integers(0, B, 2)]))
    for layout, inverse in (("interleaved", False), ("split", True)):
        y = _run(x, layout, inverse)
        ref = oracle.fft(x[rows].astype(np.complex128), inverse=inverse)
        err = rel_l2_rows(y[rows], ref)
        assert err.max() <= tol_fp32(n), (n, layout, float(err.max()))
        assert np.isfinite(y).all()


def test_plan_info_and_bytes():
    import paper_2308_00497_gb300 as fc
    p = fc.Plan(1024, 4)
    passes, radices = p.info()
    assert passes == 1 and int(np.prod(radices)) == 1024
    assert p.bytes() == 1024 * 4 * 8
    q = fc.Plan(1 << 20, 1, "split", True)
    passes, radices = q.info()   # four-step: two HBM passes
    assert passes == 2 and int(np.prod(radices)) == 1 << 20


def test_empty_batch_is_a_noop():
    import paper_2308_00497_gb300 as fc
    p = fc.Plan(256, 0)
    x = torch.empty((0, 256), dtype=torch.complex64, device="cuda")
    p.execute(x)
    torch.cuda.synchronize()


def test_misaligned_and_null_pointers():
    from paper_2308_00497_gb300 import _native as nat
    import paper_2308_00497_gb300 as fc
    lib = nat.load()
    p = fc.Plan(64, 2)
    buf = torch.zeros(2 * 64 + 4, dtype=torch.complex64, device="cuda")
    base = buf.data_ptr()
    assert lib.fftc_execute(p.handle, ctypes.c_void_p(base + 8), ctypes.c_void_p(base + 16), None) == nat.ERR_MISALIGNED
    assert lib.fftc_execute(p.handle, None, ctypes.c_void_p(base), None) == nat.ERR_INVALID_VALUE
    h = lib.fftc_plan_create(64, 2, 0, -1, 0)
    assert lib.fftc_destroy(h) == nat.OK
    assert lib.fftc_destroy(h) == nat.ERR_INVALID_PLAN   # a destroyed plan is recognised
    assert lib.fftc_execute(h, ctypes.c_void_p(base), ctypes.c_void_p(base), None) == nat.ERR_INVALID_PLAN


@pytest.mark.parametrize("layout", ["interleaved", "split"])
@pytest.mark.parametrize("inverse", [False, True])
def test_l2_resident_many_groups_ring_wrap_and_tail(monkeypatch, layout, inverse):
    """Small groups (1 MiB), a two-slot ring and a partial last group: every row checked."""
    import paper_2308_00497_gb300 as fc
    monkeypatch.setenv("FFTC_L2_RESIDENT", "1")
    monkeypatch.setenv("FFTC_L2_GROUP_MB", "1")
    monkeypatch.setenv("FFTC_L2_RING", "2")
    n, B = 1 << 16, 9          # groups of 2 transforms: 5 groups, the last one partial
    x = si.uniform_complex(B, n, seed=77)
    p = fc.Plan(n, B, layout, inverse)
    y = from_device(p.execute(to_device(x, layout)), layout)
    torch.cuda.synchronize()
    p.check()
    ref = oracle.fft(x.astype(np.complex128), inverse=inverse)
    assert rel_l2_rows(y, ref).max() <= tol_fp32(n)


@pytest.mark.parametrize("e", [15, 16, 17, 20])
def test_l2_resident_matches_two_launch_path(monkeypatch, e):
    import paper_2308_00497_gb300 as fc
    n = 1 << e
    B = max(2, (1 << 22) // n)
    x = to_device(si.uniform_complex(B, n, seed=e), "interleaved")
    monkeypatch.setenv("FFTC_L2_RESIDENT", "1")
    pa = fc.Plan(n, B)
    assert pa.info()[0] == 1
    a = pa.execute(x)
    monkeypatch.setenv("FFTC_L2_RESIDENT", "0")
    q = fc.Plan(n, B)
    assert q.info()[0] == 2
    b = q.execute(x)
    torch.cuda.synchronize()
    err = rel_l2_rows(a.cpu().numpy(), b.cpu().numpy().astype(np.complex128))
    assert err.max() <= 2 * tol_fp32(n)


@pytest.mark.parametrize("e", [15, 16, 17, 18, 19, 20])
@pytest.mark.parametrize("layout", ["interleaved", "split"])
@pytest.mark.parametrize("p2code", ["2", "6"])
def test_tensor_map_fed_four_step(monkeypatch, e, layout, p2code):
    """The bulk-copy / tensor-map fed four-step passes against the oracle: pass 1 through
    2D tensor boxes (opt-in), pass 2 refilled after its stores (2) or its last shared read (6)."""
    import paper_2308_00497_gb300 as fc
    monkeypatch.setenv("FFTC_PIPE4", "3")
    monkeypatch.setenv("FFTC_TUNE_P2_PIPE", p2code)
    n = 1 << e
    B = max(2, (1 << 21) // n)
    x = si.uniform_complex(B, n, seed=e + 5)
    p = fc.Plan(n, B, layout, e % 2 == 1)
    y = from_device(p.execute(to_device(x, layout)), layout)
    torch.cuda.synchronize()
    p.check()
    rows = np.array([0, B - 1])
    ref = oracle.fft(x[rows].astype(np.complex128), inverse=e % 2 == 1)
    assert rel_l2_rows(y[rows], ref).max() <= tol_fp32(n)


@pytest.mark.parametrize("e", [8, 9, 10, 11, 12, 13, 14])
@pytest.mark.parametrize("pipe,code", [("0", ""), ("1", ""), ("1", "2"), ("1", "6")])
def test_single_pass_both_kernels(monkeypatch, e, pipe, code):
    """Single-pass sizes through the plain kernel and the bulk-copy fed persistent kernels
    (refill after the tile's HBM stores, code 2, or after its last shared read, codes 5/6)."""
    import paper_2308_00497_gb300 as fc
    monkeypatch.setenv("FFTC_PIPE", pipe)
    monkeypatch.setenv("FFTC_TUNE_PIPE_CODE", code)
    n = 1 << e
    B = 1000 + e  # not a multiple of any tile: the last tile is partial
    x = si.uniform_complex(B, n, seed=e)
    for layout in ("interleaved", "split"):
        p = fc.Plan(n, B, layout, False)
        y = from_device(p.execute(to_device(x, layout)), layout)
        torch.cuda.synchronize()
        p.check()
        rows = np.array([0, 1, B // 2, B - 1])
        ref = oracle.fft(x[rows].astype(np.complex128))
        assert rel_l2_rows(y[rows], ref).max() <= tol_fp32(n)


@pytest.mark.parametrize("e,B", [(10, 10001), (16, 150), (20, 10), (12, 3)])
@pytest.mark.parametrize("layout", ["interleaved", "split"])
@pytest.mark.parametrize("inverse", [False, True])
def test_execute_host_chunked_matches_device_path(e, B, layout, inverse):
    """fftc_execute_host: chunked copy/transform overlap (batches above 32 MiB, ragged last
    chunk) gives bitwise the device path's result; sampled rows against the oracle."""
    import paper_2308_00497_gb300 as fc
    n = 1 << e
    x = si.uniform_complex(B, n, seed=900 + e)
    p = fc.Plan(n, B, layout, inverse)
    dev = p.execute(to_device(x, layout))
    torch.cuda.synchronize()
    xs = to_device(x, layout).cpu().pin_memory()
    out = torch.empty_like(xs).pin_memory()
    buf = torch.empty_like(xs, device="cuda")
    p.execute_host(xs, out, buf)
    assert torch.equal(out.view(torch.int32), dev.cpu().view(torch.int32))
    rows = np.array([0, B // 2, B - 1])
    y = from_device(out.cuda(), layout)
    ref = oracle.fft(x[rows].astype(np.complex128), inverse=inverse)
    assert rel_l2_rows(y[rows], ref).max() <= tol_fp32(n)


@pytest.mark.parametrize("e", [6, 10, 13, 14, 15, 18, 20])
@pytest.mark.parametrize("layout", ["interleaved", "split"])
def test_tuned_plan_matches_oracle(e, layout):
    """fftc_plan_tune swaps in the fastest compiled kernels; results stay within tolerance,
    and a second plan of the same shape reuses the cached choice."""
    import paper_2308_00497_gb300 as fc
    n = 1 << e
    B = max(3, (1 << 22) // n)
    x = si.uniform_complex(B, n, seed=e + 40)
    inverse = e % 2 == 1
    splits = set()
    for _ in range(2):
        p = fc.Plan(n, B, layout, inverse).tune(3)
        xd = to_device(x, layout)
        y1 = p.execute(xd)
        y2 = p.execute(xd)  # replay of the tuned plan: bit-identical
        torch.cuda.synchronize()
        p.check()
        assert torch.equal(y1, y2)
        y = from_device(y1, layout)
        rows = np.array([0, B // 2, B - 1])
        ref = oracle.fft(x[rows].astype(np.complex128), inverse=inverse)
        assert rel_l2_rows(y[rows], ref).max() <= tol_fp32(n)
        m, k = p.split()
        passes, radices = p.info()
        assert m * k == n and int(np.prod(radices)) == n
        if passes == 2:  # the radices of pass 1 multiply to the tuned M
            acc, i = 1, 0
            while acc < m:
                acc *= radices[i]
                i += 1
            assert acc == m
        splits.add((m, k))
    assert len(splits) == 1  # the second plan reuses the cached choice


def _timeout_then_recover(monkeypatch, n, B, layout, env):
    """Plan built with a test hook that makes every bounded device wait run out and a tiny
    poll limit: the kernel gives up, sets the plan's error word and returns, so
    fftc_plan_check reports FFTC_ERR_TIMEOUT (once: the word is cleared). A plan built
    afterwards without the hook still runs and matches the oracle."""
    import paper_2308_00497_gb300 as fc
    from paper_2308_00497_gb300 import _native as nat
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    monkeypatch.setenv("FFTC_TEST_UNREACHABLE_WAIT", "1")
    monkeypatch.setenv("FFTC_SPIN_LIMIT", "200")
    p = fc.Plan(n, B, layout)
    x = to_device(np.zeros((B, n), np.complex64), layout)
    p.execute(x)
    with pytest.raises(nat.FftcError) as ei:
        p.check()
    assert ei.value.status == nat.ERR_TIMEOUT
    p.check()
    p.close()
    monkeypatch.delenv("FFTC_TEST_UNREACHABLE_WAIT")
    monkeypatch.delenv("FFTC_SPIN_LIMIT")
    xh = si.uniform_complex(B, n, seed=77)
    q = fc.Plan(n, B, layout)
    y = from_device(q.execute(to_device(xh, layout)), layout)
    q.check()
    err = rel_l2_rows(y, oracle.fft(xh.astype(np.complex128)))
    assert err.max() <= tol_fp32(n)


@pytest.mark.parametrize("e,layout", [(12, "interleaved"), (14, "split"), (17, "interleaved"), (18, "split")])
def test_pipelined_mbarrier_wait_reports_timeout(monkeypatch, e, layout):
    """The bulk-copy fed kernels (single pass at 2^12, 2^14; four-step passes fed by bulk
    copies or tensor-map boxes at 2^17, 2^18) wait on their landing-buffer mbarriers with a
    poll limit; with the hook no copy is issued, so each wait runs out."""
    _timeout_then_recover(monkeypatch, 1 << e, 3, layout, {})


@pytest.mark.parametrize("layout", ["interleaved", "split"])
def test_l2_resident_counter_wait_reports_timeout(monkeypatch, layout):
    """The L2-resident four-step spins on per-group counters; with the hook every awaited
    count is out of reach, so each spin runs out after its poll limit."""
    _timeout_then_recover(monkeypatch, 1 << 16, 8, layout, {"FFTC_L2_RESIDENT": "1"})


@pytest.mark.parametrize("e,r", [(15, 4), (15, 2), (16, 8), (16, 4), (17, 16), (17, 8), (18, 16)])
@pytest.mark.parametrize("layout", ["interleaved", "split"])
@pytest.mark.parametrize("inverse", [False, True])
def test_cluster_single_pass(monkeypatch, e, r, layout, inverse):
    """The thread-block-cluster single pass (one HBM round trip, the middle permutation of
    Eq. 1 through distributed shared memory) for every compiled cluster shape, both layouts
    and directions, every row against the oracle; a batch that is not a multiple of the
    clusters resident at once."""
    import paper_2308_00497_gb300 as fc
    monkeypatch.setenv("FFTC_CLUSTER", "1")
    monkeypatch.setenv("FFTC_TUNE_CLUSTER_R", str(r))
    n = 1 << e
    B = 5
    x = si.uniform_complex(B, n, seed=e * 10 + r)
    p = fc.Plan(n, B, layout, inverse)
    passes, radices = p.info()
    m, k = p.split()
    assert passes == 1 and m * k == n and int(np.prod(radices)) == n
    y = from_device(p.execute(to_device(x, layout)), layout)
    torch.cuda.synchronize()
    p.check()
    ref = oracle.fft(x.astype(np.complex128), inverse=inverse)
    assert rel_l2_rows(y, ref).max() <= tol_fp32(n)


@pytest.mark.parametrize("e", [15, 16, 17, 18])
def test_cluster_full_size_and_pointwise(monkeypatch, e):
    """Sweep shape (n * batch = 2^26: many transforms per cluster) on sampled rows, in place,
    and the fused per-frequency factor of the spectral filter through the cluster pass."""
    import paper_2308_00497_gb300 as fc
    monkeypatch.setenv("FFTC_CLUSTER", "1")
    n = 1 << e
    B = (1 << 26) // n
    x = si.uniform_complex(B, n, seed=300 + e)
    rows = np.array([0, 1, B // 2, B - 1])
    p = fc.Plan(n, B)
    t = to_device(x, "interleaved")
    p.execute(t, t)
    torch.cuda.synchronize()
    p.check()
    ref = oracle.fft(x[rows].astype(np.complex128))
    assert rel_l2_rows(t[torch.from_numpy(rows).cuda()].cpu().numpy(), ref).max() <= tol_fp32(n)
    h = torch.from_numpy(si.gaussian_lowpass(n)).cuda()
    xs = to_device(x[:4], "interleaved")
    q = fc.Plan(n, 4)
    y = q.execute_pointwise(xs, h, 0.5).cpu().numpy()
    want = oracle.fft(x[:4].astype(np.complex128)) * (0.5 * si.gaussian_lowpass(n))[None, :]
    assert rel_l2_rows(y, want).max() <= tol_fp32(n)


def test_cluster_landing_wait_reports_timeout(monkeypatch):
    """The cluster pass's landing waits run out with the hook: every CTA sets the error word
    and still runs its cluster barriers, so the launch ends and the status is reported."""
    _timeout_then_recover(monkeypatch, 1 << 16, 9, "split", {"FFTC_CLUSTER": "1"})


_WISDOM_CHILD = r"""
import os, sys, json
import numpy as np
import torch
sys.path.insert(0, os.getcwd())
import paper_2308_00497_gb300 as fc
import synthetic_inputs as si
n, B = 1 << 16, 64
x = si.uniform_complex(B, n, seed=5)
p = fc.Plan(n, B).tune(2)
y = p.execute(torch.from_numpy(x).cuda())
torch.cuda.synchronize()
np.save(sys.argv[1], y.cpu().numpy())
print(json.dumps({"split": p.split(), "info": p.info()}))
"""


def _wisdom_run(tmp_path, cache, tag):
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = tmp_path / f"w_{tag}.npy"
    env = dict(os.environ, FFTC_TUNE_CACHE=str(cache))
    r = subprocess.run([sys.executable, "-c", _WISDOM_CHILD, str(out)], cwd=root, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return np.load(out), json.loads(r.stdout.strip().splitlines()[-1])


def test_tune_cache_carries_plan_choices(tmp_path):
    """FFTC_TUNE_CACHE keeps measure-mode choices across processes: the first process times the
    candidates of a 2^16 plan and appends its choice; a second process reads it back (same split
    and radices, bit-identical output); a line edited by hand to another split is honoured."""
    cache = tmp_path / "wisdom.txt"
    y1, m1 = _wisdom_run(tmp_path, cache, "first")
    lines = [ln for ln in cache.read_text().splitlines() if ln.startswith("plan ")]
    assert len(lines) == 1
    y2, m2 = _wisdom_run(tmp_path, cache, "second")
    assert m1 == m2 and np.array_equal(y1.view(np.uint32), y2.view(np.uint32))
    head, rest = lines[0].split("|", 1)
    f = rest.split()
    assert f[5] in ("S", "F", "C")
    # a two-pass choice at the split 2^7 x 2^9 (plain column kernel: E 16, 16 lines, runtime
    # stride; row kernel: E 32, 16 lines, runtime stride), appended after the first line
    other = f"{head}|{' '.join(f[:5])} F 7 0 1 7 4 16 0 0 0 0 0 2 9 5 16 0 0 0 0 0"
    with open(cache, "a") as fh:
        fh.write(other + "\n")
    y3, m3 = _wisdom_run(tmp_path, cache, "edited")
    assert tuple(m3["split"]) == (128, 512)
    x = si.uniform_complex(64, 1 << 16, seed=5)
    ref = oracle.fft(x[[0, 63]].astype(np.complex128))
    assert rel_l2_rows(y3[[0, 63]], ref).max() <= tol_fp32(1 << 16)


@pytest.mark.parametrize("e,logm,loge,lines,p1", [
    (15, 7, 4, 32, 0), (16, 8, 4, 32, 0), (17, 8, 4, 32, 0), (16, 8, 5, 32, 0), (17, 8, 5, 32, 0),
    (15, 7, 4, 32, 5), (16, 8, 4, 32, 5), (17, 8, 4, 32, 5),
    (20, 9, 4, 16, 5), (20, 9, 4, 32, 5), (20, 10, 4, 16, 5), (20, 10, 5, 8, 5),
    (19, 9, 5, 32, 0), (20, 9, 5, 32, 0), (19, 9, 4, 32, 5), (20, 9, 4, 16, 0), (20, 9, 5, 16, 0),
])
@pytest.mark.parametrize("layout", ["interleaved", "split"])
def test_pass1_band_variants(monkeypatch, e, logm, loge, lines, p1, layout):
    """Every pass-1 column kernel that measure-mode planning may pick for the sweep sizes (plain
    loads or tensor-map boxes, 8 to 32 columns, 16 or 32 elements per thread), forced through
    the planner's knobs, against the oracle on sampled rows."""
    import paper_2308_00497_gb300 as fc
    monkeypatch.setenv("FFTC_TUNE_FOURSTEP_LOGM", str(logm))
    monkeypatch.setenv("FFTC_TUNE_COLS_E", str(loge))
    monkeypatch.setenv("FFTC_TUNE_COLS_C", str(lines))
    monkeypatch.setenv("FFTC_PIPE4", "1" if p1 else "0")
    if p1:
        monkeypatch.setenv("FFTC_TUNE_P1_PIPE", str(p1))
    n = 1 << e
    B = max(3, (1 << 22) // n)
    x = si.uniform_complex(B, n, seed=e * 7 + lines)
    p = fc.Plan(n, B, layout, e % 2 == 0)
    assert p.split()[0] == 1 << logm
    assert p.info()[1][0] == 1 << loge  # pass 1 runs radix-2^loge stages
    y = from_device(p.execute(to_device(x, layout)), layout)
    torch.cuda.synchronize()
    p.check()
    rows = np.array([0, B // 2, B - 1])
    ref = oracle.fft(x[rows].astype(np.complex128), inverse=e % 2 == 0)
    assert rel_l2_rows(y[rows], ref).max() <= tol_fp32(n)


@pytest.mark.parametrize("layout", ["interleaved", "split"])
@pytest.mark.parametrize("inverse", [False, True])
def test_2p20_pass2_bulk_copy_compile_time_stride(monkeypatch, layout, inverse):
    """n = 2^20 split as 2^9 x 2^11 with pass 2 fed by one bulk copy per tile of 8 rows of
    2048 points and its transposed store at the compile-time stride 2^9, against the oracle
    on sampled rows."""
    import paper_2308_00497_gb300 as fc
    for k, v in (("FFTC_TUNE_FOURSTEP_LOGM", 9), ("FFTC_TUNE_ROWST_E", 5), ("FFTC_TUNE_ROWST_C", 8),
                 ("FFTC_PIPE4", 2), ("FFTC_TUNE_P2_PIPE", 5)):
        monkeypatch.setenv(k, str(v))
    n, B = 1 << 20, 5
    x = si.uniform_complex(B, n, seed=91)
    p = fc.Plan(n, B, layout, inverse)
    assert p.split() == (512, 2048)
    y = from_device(p.execute(to_device(x, layout)), layout)
    torch.cuda.synchronize()
    p.check()
    rows = np.array([0, B - 1])
    ref = oracle.fft(x[rows].astype(np.complex128), inverse=inverse)
    assert rel_l2_rows(y[rows], ref).max() <= tol_fp32(n)


@pytest.mark.parametrize("e,logm,logk", [(17, 8, 9), (18, 8, 10), (19, 9, 10)])
@pytest.mark.parametrize("inverse", [False, True])
def test_split_pass2_16_row_tiles(monkeypatch, e, logm, logk, inverse):
    """Split-layout output through the bulk-copy fed pass 2 with 16-row tiles (16 consecutive
    outputs per plane in each transposed store), against the oracle on sampled rows."""
    import paper_2308_00497_gb300 as fc
    for k, v in (("FFTC_TUNE_FOURSTEP_LOGM", logm), ("FFTC_TUNE_ROWST_E", 5), ("FFTC_TUNE_ROWST_C", 16),
                 ("FFTC_PIPE4", 2), ("FFTC_TUNE_P2_PIPE", 5)):
        monkeypatch.setenv(k, str(v))
    n = 1 << e
    B = max(3, (1 << 22) // n)
    x = si.uniform_complex(B, n, seed=e + 300)
    p = fc.Plan(n, B, "split", inverse)
    assert p.split() == (1 << logm, 1 << logk)
    y = from_device(p.execute(to_device(x, "split")), "split")
    torch.cuda.synchronize()
    p.check()
    rows = np.array([0, B // 2, B - 1])
    ref = oracle.fft(x[rows].astype(np.complex128), inverse=inverse)
    assert rel_l2_rows(y[rows], ref).max() <= tol_fp32(n)

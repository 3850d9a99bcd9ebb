"""Uneven batches in one persistent launch (graph replay): parity with the oracle,
determinism, buffer switching, and the bounded-wait error path (made to time out on
purpose with a dependency nothing satisfies; the GPU context stays usable)."""
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


def _check_rows(x, y, n, d, o, rows):
    for i in rows:
        xi = x[o[i]:o[i] + n[i]].astype(np.complex128)
        ref = oracle.fft(xi, inverse=d[i] == 1)
        err = rel_l2_rows(y[o[i]:o[i] + n[i]][None], ref[None])[0]
        assert err <= tol_fp32(int(n[i])), (i, int(n[i]), float(err))


def test_small_uneven_batch_all_rows():
    import paper_2308_00497_gb300 as fc
    rng = np.random.default_rng(3)
    e = np.concatenate([np.arange(6, 17), rng.integers(6, 17, 29)])
    n = (1 << e).astype(np.int64)
    d = np.where(rng.random(n.size) < 0.5, -1, 1).astype(np.int8)
    gaps = rng.integers(0, 3, n.size) * 16          # rows need not be packed
    o = np.concatenate([[0], np.cumsum(n + gaps)[:-1]]).astype(np.int64)
    total = int(o[-1] + n[-1])
    x = si.uniform_complex(1, total, seed=9).reshape(total)
    p = fc.UnevenPlan(n, d, o)
    xd = torch.from_numpy(x).cuda()
    yd = torch.zeros_like(xd)
    p.execute(xd, yd)
    torch.cuda.synchronize()
    p.check()
    _check_rows(x, yd.cpu().numpy(), n, d, o, range(n.size))


def test_workload_4096_sampled_and_deterministic():
    import paper_2308_00497_gb300 as fc
    n, d, o, total = si.uneven_batch(4096, seed=4)
    x = si.uneven_data(total, seed=4)
    p = fc.UnevenPlan(n, d, o)
    xd = torch.from_numpy(x).cuda()
    y1 = torch.empty_like(xd)
    p.execute(xd, y1)
    y2 = p.execute(xd)              # another output buffer: the graph's node is updated
    y3 = torch.empty_like(xd)
    p.execute(xd, y3)
    torch.cuda.synchronize()
    p.check()
    assert torch.equal(y1.view(torch.float32), y2.view(torch.float32))
    assert torch.equal(y1.view(torch.float32), y3.view(torch.float32))
    rng = np.random.default_rng(1)
    rows = []
    for lg in range(6, 17):        # three rows of every length, both directions present
        idx = np.flatnonzero(n == (1 << lg))
        rows += list(rng.choice(idx, size=min(3, idx.size), replace=False))
    _check_rows(x, y1.cpu().numpy(), n, d, o, rows)


def test_in_place_uneven():
    import paper_2308_00497_gb300 as fc
    n, d, o, total = si.uneven_batch(200, seed=5)
    x = si.uneven_data(total, seed=5)
    p = fc.UnevenPlan(n, d, o)
    xd = torch.from_numpy(x).cuda()
    p.execute(xd, xd)
    torch.cuda.synchronize()
    _check_rows(x, xd.cpu().numpy(), n, d, o, range(0, 200, 7))


def test_bounded_wait_reports_timeout(monkeypatch):
    """Pass-2 tiles wait for a count nothing reaches; with a tiny spin limit every wait
    gives up, the kernel returns, and fftc_plan_check reports FFTC_ERR_TIMEOUT."""
    import paper_2308_00497_gb300 as fc
    from paper_2308_00497_gb300 import _native as nat
    monkeypatch.setenv("FFTC_TEST_UNREACHABLE_WAIT", "1")
    monkeypatch.setenv("FFTC_SPIN_LIMIT", "200")
    n = np.array([1 << 14, 1 << 13, 256], dtype=np.int64)
    d = np.array([-1, 1, -1], dtype=np.int8)
    o = np.array([0, 1 << 14, 3 << 13], dtype=np.int64)
    p = fc.UnevenPlan(n, d, o)
    x = torch.zeros(int(o[-1] + n[-1]), dtype=torch.complex64, device="cuda")
    p.execute(x)
    with pytest.raises(nat.FftcError) as ei:
        p.check()
    assert ei.value.status == nat.ERR_TIMEOUT
    p.check()  # the error word was cleared
    monkeypatch.delenv("FFTC_TEST_UNREACHABLE_WAIT")
    monkeypatch.delenv("FFTC_SPIN_LIMIT")
    q = fc.UnevenPlan(n, d, o)  # the context is still usable
    y = q.execute(torch.ones_like(x))
    torch.cuda.synchronize()
    q.check()
    assert torch.isfinite(y.view(torch.float32)).all()


# every compiled four-step configuration of the classes 2^13 .. 2^16: (log2 n, log2 M, variant)
# with variant 0 = 2^(L - 4) elements per thread, 16 lines a tile; 1 = half of them; 2 = 16
# elements per thread on every line length (4096-element tiles)
FOUR_STEP_CONFIGS = [(13, 6, 0), (13, 7, 0), (14, 7, 0), (15, 7, 0), (15, 8, 0), (16, 8, 0),
                     (14, 7, 1), (15, 7, 1), (15, 8, 1), (16, 8, 1),
                     (13, 6, 2), (13, 7, 2), (14, 6, 2), (14, 7, 2), (14, 8, 2), (15, 7, 2), (15, 8, 2)]


@pytest.mark.parametrize("logn,logm,ev", FOUR_STEP_CONFIGS)
def test_every_four_step_branch(monkeypatch, logn, logm, ev):
    """Each four-step split and tile shape the autotuner may pick for a length class, forced
    through its override, on rows of both directions beside a single-pass class; every row
    against the oracle."""
    import paper_2308_00497_gb300 as fc
    monkeypatch.setenv(f"FFTC_UNEVEN_LOGM_{logn}", str(logm))
    monkeypatch.setenv(f"FFTC_UNEVEN_EV_{logn}", str(ev))
    n = np.array([1 << logn] * 5 + [256] * 3, dtype=np.int64)
    d = np.array([-1, 1, -1, 1, 1, -1, 1, -1], dtype=np.int8)
    o = np.concatenate([[0], np.cumsum(n)[:-1]]).astype(np.int64)
    total = int(o[-1] + n[-1])
    x = si.uniform_complex(1, total, seed=40 + logn + 3 * logm + ev).reshape(total)
    p = fc.UnevenPlan(n, d, o)
    y = p.execute(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    p.check()
    _check_rows(x, y.cpu().numpy(), n, d, o, range(n.size))


def test_uneven_rejects_bad_descriptors():
    import paper_2308_00497_gb300 as fc
    from paper_2308_00497_gb300 import _native as nat
    with pytest.raises(nat.FftcError) as ei:   # overlapping rows
        fc.UnevenPlan(np.array([64, 64]), np.array([-1, -1]), np.array([0, 32]))
    assert ei.value.status == nat.ERR_INVALID_VALUE


_CACHE_CHILD = r"""
import os, sys
import numpy as np
import torch
sys.path.insert(0, os.getcwd())
import paper_2308_00497_gb300 as fc
import synthetic_inputs as si
n = np.array([1 << 13] * 3 + [1 << 15] * 3 + [256] * 5, dtype=np.int64)
d = np.array([-1, 1, -1, 1, -1, 1, -1, 1, -1, 1, -1], dtype=np.int8)
o = np.concatenate([[0], np.cumsum(n)[:-1]]).astype(np.int64)
total = int(o[-1] + n[-1])
x = si.uniform_complex(1, total, seed=31).reshape(total)
p = fc.UnevenPlan(n, d, o)
y = p.execute(torch.from_numpy(x).cuda())
torch.cuda.synchronize()
p.check()
np.save(sys.argv[1], y.cpu().numpy())
"""


def _cache_run(tmp_path, cache, tag):
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = tmp_path / f"y_{tag}.npy"
    env = dict(os.environ, FFTC_TUNE="1", FFTC_TUNE_CACHE=str(cache))
    r = subprocess.run([sys.executable, "-c", _CACHE_CHILD, str(out)], cwd=root, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return np.load(out)


def test_tune_cache_file_round_trip(tmp_path):
    """FFTC_TUNE_CACHE carries the autotuner's per-class choices across processes: a first
    process times the candidate splits of the 2^13 and 2^15 classes and appends its choices;
    a second process reads them back and builds the same plan (bit-identical output); an
    entry appended to the file by hand is honoured (another split: different rounding,
    still within tolerance of the oracle)."""
    cache = tmp_path / "tune.txt"
    y1 = _cache_run(tmp_path, cache, "first")
    # "uneven <device name>|<log2 n> <log2 M, 0 for one pass> <tile variant: 0, 1 half, 2 wide>"
    lines = [ln.split() for ln in cache.read_text().splitlines() if ln.startswith("uneven ")]
    chosen = {int(t[-3].split("|")[-1]): (int(t[-2]), int(t[-1])) for t in lines}
    assert {13, 15} <= set(chosen)
    y2 = _cache_run(tmp_path, cache, "second")
    assert np.array_equal(y1.view(np.uint32), y2.view(np.uint32))
    dev = " ".join(lines[0][1:-2]).rsplit("|", 1)[0]
    other = 8 if chosen[15][0] == 7 else 7
    with open(cache, "a") as f:
        f.write(f"uneven {dev}|15 {other} 0\n")
    y3 = _cache_run(tmp_path, cache, "edited")
    n = np.array([1 << 13] * 3 + [1 << 15] * 3 + [256] * 5, dtype=np.int64)
    d = np.array([-1, 1, -1, 1, -1, 1, -1, 1, -1, 1, -1], dtype=np.int8)
    o = np.concatenate([[0], np.cumsum(n)[:-1]]).astype(np.int64)
    total = int(o[-1] + n[-1])
    x = si.uniform_complex(1, total, seed=31).reshape(total)
    _check_rows(x, y3, n, d, o, range(len(n)))
    r15 = slice(int(o[3]), int(o[6]))
    assert not np.array_equal(y1[r15].view(np.uint32), y3[r15].view(np.uint32))

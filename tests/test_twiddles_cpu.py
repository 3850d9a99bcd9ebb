"""Pin of the twiddle diagonals D (Eq. 1; Table 1 "Mul"): every FP32 entry the library
uploads is the round-to-nearest float of the FP64 root of unity w_{Ns R}^{t k}, computed
here independently with numpy from the definition (no library code involved)."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2308_00497_gb300 import _native, build
    build.build()
    return _native.load()


def schedule(logl, loge):
    """Radix schedule: stages of radix 2^loge, the remainder radix last; Ns = product before."""
    S = (logl + loge - 1) // loge
    rem = logl % loge
    lr = [rem if (rem and s == S - 1) else loge for s in range(S)]
    lns = [sum(lr[:s]) for s in range(S)]
    return lr, lns


def expected(logl, loge):
    lr, lns = schedule(logl, loge)
    out = []
    for s in range(1, len(lr)):
        R, Ns = 1 << lr[s], 1 << lns[s]
        L = Ns * R
        t = np.arange(1, R)[:, None]
        k = np.arange(Ns)[None, :]
        m = (t * k) % L
        ang = 2.0 * np.pi * m / L
        w = np.cos(ang) - 1j * np.sin(ang)
        # at quarter turns the exact root is 1, -i, -1 or +i (FP64 cos(pi/2) is not 0)
        q = (4 * m) % L == 0
        w[q] = np.array([1, -1j, -1, 1j])[(4 * m[q]) // L]
        out.append(w.reshape(-1))
    return np.concatenate(out) if out else np.zeros(0, complex)


@pytest.mark.parametrize("logl,loge", [(4, 4), (8, 4), (10, 5), (12, 4), (13, 5), (11, 4), (10, 3), (16, 4),
                                       (20, 5), (7, 3)])
def test_tables_are_rounded_fp64_roots(lib, logl, loge):
    want = expected(logl, loge)
    buf = np.zeros(2 * max(1, want.size), np.float32)
    cnt = ctypes.c_int64(0)
    assert lib.fftc_stage_twiddles(logl, loge, buf.ctypes.data, buf.size // 2, ctypes.byref(cnt)) == 0
    assert cnt.value == want.size
    got = buf[: 2 * want.size].reshape(-1, 2)
    wr = want.real.astype(np.float32)
    wi = want.imag.astype(np.float32)
    # exact except where numpy's FP64 value and the library's octant-reduced one straddle a
    # float rounding boundary; then they differ by one float ulp at most
    if want.size == 0:  # a single stage has no twiddles
        return
    exact = (got[:, 0] == wr) & (got[:, 1] == wi)
    assert exact.mean() > 0.999
    ulp_r = np.abs(np.spacing(wr))
    ulp_i = np.abs(np.spacing(wi))
    assert np.all(np.abs(got[:, 0] - wr) <= ulp_r) and np.all(np.abs(got[:, 1] - wi) <= ulp_i)


def test_special_entries_exact(lib):
    """Entries with t k = 0, L/8 and L/4 are 1, (1 - i)/sqrt2 rounded, and -i exactly."""
    buf = np.zeros(2 * 4096, np.float32)
    cnt = ctypes.c_int64(0)
    assert lib.fftc_stage_twiddles(8, 4, buf.ctypes.data, 4096, ctypes.byref(cnt)) == 0
    t = buf[: 2 * cnt.value].reshape(15, 16, 2)  # stage 1: R = 16, Ns = 16, L = 256; row t-1, column k
    assert tuple(t[0, 0]) == (1.0, 0.0)                       # t k = 0
    h = np.float32(np.sqrt(0.5))
    assert tuple(t[3, 8]) == (h, -h)                          # t k = 32 = L/8
    assert tuple(t[7, 8]) == (0.0, -1.0)                      # t k = 64 = L/4


def test_bad_arguments(lib):
    cnt = ctypes.c_int64(0)
    assert lib.fftc_stage_twiddles(3, 4, None, 0, ctypes.byref(cnt)) != 0
    assert lib.fftc_stage_twiddles(21, 4, None, 0, ctypes.byref(cnt)) != 0
    buf = np.zeros(2, np.float32)
    assert lib.fftc_stage_twiddles(10, 5, buf.ctypes.data, 1, ctypes.byref(cnt)) != 0  # too small
    assert cnt.value == 31 * 32


def test_odd_radix_constants_in_the_mixed_kernel():
    """The cos / sin literals of the radix-3, -5 and -7 butterflies are cos(2 pi m / r)
    and sin(2 pi m / r) (checked against the C library in FP64, then FP32 rounding)."""
    import math
    import os
    import re
    src = open(os.path.join(os.path.dirname(__file__), "..", "paper_2308_00497_gb300", "csrc",
                            "fftc_mixed.cuh")).read()

    def table(fn):
        body = src[src.index(f"constexpr float {fn}(int r, int m)"):]
        body = body[:body.index("}")]
        return [float(v) for v in re.findall(r"(-?\d+\.\d+)f", body)]

    cos_vals, sin_vals = table("mixed_cos"), table("mixed_sin")
    # literal order in the source: r = 3 (m = 1, twice), r = 5 (m = 1, 2), r = 7 (m = 1, 2, 3)
    want_cos = [math.cos(2 * math.pi / 3)] * 2 + [math.cos(2 * math.pi * m / 5) for m in (1, 2)] + \
               [math.cos(2 * math.pi * m / 7) for m in (1, 2, 3)]
    want_sin = [math.sin(2 * math.pi / 3)] + [math.sin(2 * math.pi * m / 5) for m in (1, 2)] + \
               [math.sin(2 * math.pi * m / 7) for m in (1, 2, 3)]
    assert len(cos_vals) == len(want_cos) and len(sin_vals) == len(want_sin)
    for got, want in zip(cos_vals + sin_vals, want_cos + want_sin):
        assert abs(got - want) <= 1e-15, (got, want)


def test_compile_time_trig_of_the_composite_butterflies(tmp_path):
    """ct_cos / ct_sin (fftc_ctrig.h, the constants inside the composite-radix butterflies)
    equal cos / sin(2 pi m / N) to 1e-15 for every N <= 32 and m < N."""
    import math
    import os
    import subprocess
    hdr = os.path.abspath(os.path.join(os.path.dirname(__file__), "..", "paper_2308_00497_gb300", "csrc"))
    src = tmp_path / "t.cpp"
    src.write_text('#include <cstdio>\n#include "fftc_ctrig.h"\nint main(){for(int N=1;N<=32;++N)'
                   'for(int m=-N;m<2*N;++m)std::printf("%d %d %.17g %.17g\\n",m,N,fftc::ct_cos(m,N),'
                   'fftc::ct_sin(m,N));}\n')
    exe = tmp_path / "t"
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", hdr, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    rows = [ln.split() for ln in out if ln]
    assert len(rows) == sum(3 * N for N in range(1, 33))
    for m, N, c, s in rows:
        # reference angle folded into [0, pi] exactly first (the argument rounding of an
        # unfolded 2 pi m / N near 2 pi alone costs ~1e-15)
        mm, n = int(m) % int(N), int(N)
        k, sgn = (n - mm, -1.0) if 2 * mm > n else (mm, 1.0)
        ang = 2 * math.pi * k / n
        assert abs(float(c) - math.cos(ang)) <= 1e-15 and abs(float(s) - sgn * math.sin(ang)) <= 1e-15, (m, N)

"""fftc_execute_noalloc: the allocation-free two-pass transform for callers that may
not allocate device memory (a plugin whose host application owns the GPU memory
budget, a loop that forbids allocation after start-up).

Called through the C ABI, its output must match the plan-based entry point
(fftc_execute) on the same input within the FP32 tolerance of the other tests,
on two calls in a row (the second one reuses the shared scratch array, which
then holds the first call's data), and sampled rows must match the FP64 oracle
within the same tolerance, so that the result stands on its own and not only
against the library's other path. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synthetic_inputs as si
from gpu_util import from_device, rel_l2_rows, to_device, tol_fp32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2308_00497_gb300 import _native, build
    build.build()
    return _native.load()


@pytest.mark.parametrize("e,batch,layout,inverse", [
    (14, 64, "interleaved", False),
    (15, 8, "split", False),
    (16, 32, "split", True),
    (17, 3, "split", False),
    (18, 8, "interleaved", True),
    (19, 4, "split", True),
    (20, 2, "interleaved", True),
])
def test_noalloc_matches_plan_and_oracle_two_calls(lib, e, batch, layout, inverse):
    from paper_2308_00497_gb300 import _native as nat
    import paper_2308_00497_gb300 as fc
    n = 1 << e
    plan = fc.Plan(n, batch, layout, inverse)
    stream = torch.cuda.current_stream().cuda_stream
    rows = sorted({0, batch - 1})
    for call, seed in enumerate((11, 12)):  # two calls in a row, different data
        xh = si.uniform_complex(batch, n, seed=seed + e)
        x = to_device(xh, layout)
        ref = plan.execute(x)
        out = torch.empty_like(x)
        st = lib.fftc_execute_noalloc(n, batch, nat.LAYOUTS[layout], nat.INVERSE if inverse else nat.FORWARD,
                                      ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(stream))
        assert st == nat.OK, nat.status_string(st)
        torch.cuda.synchronize()
        got = from_device(out, layout)
        err = rel_l2_rows(got, from_device(ref, layout).astype(np.complex128))
        assert err.max() <= tol_fp32(n), (call, float(err.max()))
        want = oracle.fft(xh[rows].astype(np.complex128), inverse=inverse)
        err_o = rel_l2_rows(got[rows], want)
        assert err_o.max() <= tol_fp32(n), (call, float(err_o.max()))


def test_noalloc_rejects_out_of_range(lib):
    from paper_2308_00497_gb300 import _native as nat
    buf = torch.zeros(16, dtype=torch.complex64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    assert lib.fftc_execute_noalloc(1 << 13, 1, 0, -1, p, p, None) == nat.ERR_UNSUPPORTED_SIZE   # needs no workspace
    assert lib.fftc_execute_noalloc(1 << 21, 1, 0, -1, p, p, None) == nat.ERR_UNSUPPORTED_SIZE
    assert lib.fftc_execute_noalloc(1 << 20, 3, 0, -1, p, p, None) == nat.ERR_UNSUPPORTED_SIZE   # > scratch capacity
    assert lib.fftc_execute_noalloc(1 << 14, -1, 0, -1, p, p, None) == nat.ERR_INVALID_VALUE
    assert lib.fftc_execute_noalloc(1 << 14, 0, 0, -1, p, p, None) == nat.OK
    assert lib.fftc_execute_noalloc(1 << 14, 1, 0, -1, ctypes.c_void_p(buf.data_ptr() + 8), p, None) == nat.ERR_MISALIGNED

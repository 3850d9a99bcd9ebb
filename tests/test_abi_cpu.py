"""The C ABI loads and exports every symbol include/fftc.h declares; argument
validation that needs no device (bad sizes, bad enums, NULL and stale plans)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fftc.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2308_00497_gb300 import build, _native
    build.build()
    return _native.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fftc_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name


def test_binding_declares_every_symbol(lib):
    from paper_2308_00497_gb300 import _native
    assert set(declared_functions()) == set(_native.PROTOTYPES)


def test_status_strings(lib):
    from paper_2308_00497_gb300 import _native as nat
    names = [nat.status_string(i) for i in range(8)]
    assert names[0] == "FFTC_OK" and names[7] == "FFTC_ERR_TIMEOUT"
    assert len(set(names)) == 8
    assert nat.status_string(99) == "FFTC_ERR_UNKNOWN"


@pytest.mark.parametrize("n", [0, 1, 11, 22, 143, 1 << 25, 3 << 23, 7 * (1 << 22), -8])
def test_unsupported_sizes_rejected_before_any_device_call(lib, n):
    """Lengths outside [2, 2^24] or with a prime factor above 7."""
    from paper_2308_00497_gb300 import _native as nat
    assert not lib.fftc_plan_create(n, 4, 0, -1, 0)
    assert lib.fftc_get_last_error() == nat.ERR_UNSUPPORTED_SIZE


def _splits(n, line):
    return n <= line or any(n % m == 0 and n // m <= line for m in range(2, line + 1))


@pytest.mark.parametrize("n", [9565938, 12907776])
def test_fp64_lengths_without_a_two_factor_split_rejected(lib, n):
    """FP64 runs lines of at most 4096 points: above that n needs n = M K with M, K <= 4096.
    These 7-smooth lengths below 2^24 have none (a brute-force divisor search says so),
    while FP32 lines of 8192 split them."""
    from paper_2308_00497_gb300 import _native as nat
    assert not _splits(n, 4096) and _splits(n, 8192)
    assert not lib.fftc_plan_create(n, 4, 0, -1, nat.FP64)
    assert lib.fftc_get_last_error() == nat.ERR_UNSUPPORTED_SIZE


@pytest.mark.parametrize("precision", [1, 2, 3, 4])
def test_mixed_radix_sizes_are_fp32_only(lib, precision):
    from paper_2308_00497_gb300 import _native as nat
    assert not lib.fftc_plan_create(12, 4, 0, -1, precision)
    assert lib.fftc_get_last_error() == nat.ERR_UNSUPPORTED_SIZE


@pytest.mark.parametrize("args", [(64, -1, 0, -1, 0), (64, 4, 2, -1, 0), (64, 4, 0, 0, 0), (64, 4, 0, -1, 9)])
def test_bad_arguments_rejected(lib, args):
    from paper_2308_00497_gb300 import _native as nat
    assert not lib.fftc_plan_create(*args)
    assert lib.fftc_get_last_error() == nat.ERR_INVALID_VALUE


def test_null_and_foreign_plans(lib):
    from paper_2308_00497_gb300 import _native as nat
    assert lib.fftc_destroy(None) == nat.OK
    bogus = ctypes.c_void_p(0x1000)
    assert lib.fftc_destroy(bogus) == nat.ERR_INVALID_PLAN
    assert lib.fftc_execute(None, None, None, None) == nat.ERR_INVALID_PLAN
    assert lib.fftc_execute(bogus, None, None, None) == nat.ERR_INVALID_PLAN
    assert lib.fftc_plan_bytes(bogus) == 0
    assert lib.fftc_plan_info(bogus, None, None, None) == nat.ERR_INVALID_PLAN
    assert lib.fftc_plan_check(None, None) == nat.ERR_INVALID_PLAN


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2308_00497_gb300 import _native as nat
    monkeypatch.setattr(nat, "_lib", None)
    monkeypatch.setattr(nat, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        nat.load()


def test_uneven_validation_before_any_device_call(lib):
    import numpy as np
    from paper_2308_00497_gb300 import _native as nat
    n = np.array([64, 32], dtype=np.int64)
    d = np.array([-1, 1], dtype=np.int8)
    o = np.array([0, 64], dtype=np.int64)
    assert not lib.fftc_plan_create_uneven(2, n.ctypes.data, d.ctypes.data, o.ctypes.data, 0, 0)
    assert lib.fftc_get_last_error() == nat.ERR_UNSUPPORTED_SIZE       # 32 < 64
    assert not lib.fftc_plan_create_uneven(0, n.ctypes.data, d.ctypes.data, o.ctypes.data, 0, 0)
    assert lib.fftc_get_last_error() == nat.ERR_INVALID_VALUE
    assert not lib.fftc_plan_create_uneven(1, n.ctypes.data, d.ctypes.data, o.ctypes.data, 1, 0)
    assert lib.fftc_get_last_error() == nat.ERR_INVALID_VALUE          # split layout


@pytest.mark.parametrize("dims", [(16384, 4), (11, 16), (4, 22), (1, 8), (8, 1 << 25)])
def test_nd_unsupported_shapes_rejected_before_any_device_call(lib, dims):
    import ctypes
    from paper_2308_00497_gb300 import _native as nat
    arr = (ctypes.c_int64 * len(dims))(*dims)
    assert not lib.fftc_plan_create_nd(len(dims), arr, 2, 0, -1, 0)
    assert lib.fftc_get_last_error() == nat.ERR_UNSUPPORTED_SIZE


def test_nd_bad_arguments_rejected(lib):
    import ctypes
    from paper_2308_00497_gb300 import _native as nat
    arr = (ctypes.c_int64 * 4)(8, 8, 8, 8)
    for args in ((1, arr, 2, 0, -1, 0), (4, arr, 2, 0, -1, 0), (2, None, 2, 0, -1, 0), (2, arr, -1, 0, -1, 0),
                 (2, arr, 2, 5, -1, 0), (2, arr, 2, 0, 3, 0)):
        assert not lib.fftc_plan_create_nd(*args)
        assert lib.fftc_get_last_error() == nat.ERR_INVALID_VALUE
    assert not lib.fftc_plan_create_nd(2, arr, 2, 0, -1, 1)  # tensor-core precisions: 1D only
    assert lib.fftc_get_last_error() == nat.ERR_UNSUPPORTED_SIZE


def test_tune_rejects_null_plan_and_bad_reps(lib):
    from paper_2308_00497_gb300 import _native as nat
    assert lib.fftc_plan_tune(None, 3) == nat.ERR_INVALID_PLAN

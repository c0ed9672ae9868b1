"""C-ABI checks that need no GPU: the library loads, exports every function
include/tcfft.h declares, and rejects bad arguments before touching a device."""
import ctypes
import os
import re

import pytest

import paper_2104_11471_gb300 as tc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tcfft.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tcfft_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    tc.build()
    return tc.lib()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "tcfft_plan_1d" in names and "tcfft_exec" in names and "tcfft_destroy" in names
    for name in names:
        assert hasattr(lib, name), name
        assert name in tc._SIG, f"binding lacks {name}"


def test_status_strings(lib):
    for code, name in tc.STATUS.items():
        assert tc.tcfft_status_string(code) == name
    assert tc.tcfft_status_string(99) == "TCFFT_ERR_UNKNOWN"


def test_argument_checks_before_device(lib):
    h = ctypes.c_void_p()
    assert lib.tcfft_plan_1d(None, 256, 1) == 2
    for n, b in ((100, 1), (8, 1), (1 << 28, 1), (256, 0), (256, -3)):
        assert lib.tcfft_plan_1d(ctypes.byref(h), n, b) == 1, (n, b)
    for nx, ny in ((16, 8), (8192 * 2, 16), (48, 64)):
        assert lib.tcfft_plan_2d(ctypes.byref(h), nx, ny, 1) == 1
    assert lib.tcfft_plan_1d_ex(ctypes.byref(h), 256, 1, 7, 0) == 2   # bad precision
    assert lib.tcfft_plan_1d_ex(ctypes.byref(h), 256, 1, 0, 1 << 10) == 2  # unknown flag bit
    a = (ctypes.c_int64 * 2)(256, 100)
    assert lib.tcfft_plan_many(ctypes.byref(h), 2, a, None, 0, 0) == 1  # 100 is not a power of two
    b = (ctypes.c_int64 * 1)(1 << 25)
    assert lib.tcfft_plan_many(ctypes.byref(h), 1, b, None, 0, 0) == 1  # ragged 1D stops at 2^24
    assert lib.tcfft_plan_many(ctypes.byref(h), 0, a, None, 0, 0) == 1
    assert lib.tcfft_plan_many(ctypes.byref(h), 2, None, None, 0, 0) == 2
    assert lib.tcfft_exec(None, None, None, None) == 2
    assert lib.tcfft_destroy(None) == 0
    assert lib.tcfft_io_bytes(None) == 0


def test_binding_raises_without_device_or_on_bad_size(lib):
    import torch
    with pytest.raises(tc.TcfftError) as e:
        tc.tcfft_plan_1d(100, 1)
    assert e.value.status == 1
    if not torch.cuda.is_available():
        with pytest.raises(tc.TcfftError) as e:
            tc.tcfft_plan_1d(256, 1)
        assert e.value.status == 6  # no sm_103a device: unsupported, never a CPU fallback

"""The allocation-free entry point tcfft_exec_1d_noalloc.

tcfft_exec_1d_noalloc serves callers that cannot allocate device memory when
they need a transform (a process that reserved its device-memory budget up
front, or a loop that must not pay for cudaMalloc/cudaFree).  It keeps its
workspace in a fixed device array shared by all calls, so these tests run
calls of different sizes in a row and check each one:
  * against tcfft_plan_1d + tcfft_exec on the same input, bit for bit where
    both run the same two passes (2^15 .. 2^21; the plans switch to three
    passes from 2^22), within the tolerance of the other tests elsewhere;
  * against the FP64 oracle (rel-L2 and the per-element bound), including
    the two-pass splits 2048 x 2048 .. 4096 x 4096 that only this entry point
    runs (2^22 .. 2^24) and in-place calls.
This file is collected last on purpose; it must pass both alone in a fresh
process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import oracle
import seeded_inputs as si
from gpu_helpers import PLAIN_TOL, check_rows, to_device

pytestmark = pytest.mark.gpu


def _run_plan(n, batch, x):
    import torch
    import paper_2104_11471_gb300 as tc
    y = torch.full_like(x, 0x7E00)
    plan = tc.Plan.plan_1d(n, batch)
    plan.exec(x, y)
    torch.cuda.synchronize()
    assert plan.last_error() == 0
    plan.destroy()
    return y


def _noalloc(n, batch, x, y):
    import torch
    import paper_2104_11471_gb300 as tc
    stream = torch.cuda.current_stream().cuda_stream
    st = tc.lib().tcfft_exec_1d_noalloc(ctypes.c_int64(n), ctypes.c_int64(batch), ctypes.c_void_p(x.data_ptr()),
                                        ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(stream))
    assert st == 0, tc.STATUS.get(st)
    torch.cuda.synchronize()


def _c(t, batch, n):
    return si.as_complex128(t.cpu().numpy().view(np.float16).reshape(batch, n, 2))


def test_noalloc_matches_plan_path_two_calls():
    import torch
    for n, batch, seed in ((1 << 20, 3, 71), (1 << 16, 5, 72), (1 << 21, 2, 73)):
        h = si.half_input((batch, n), seed=seed)
        x = to_device(h)
        ref = _run_plan(n, batch, x)
        y = torch.full_like(x, 0x7E00)
        _noalloc(n, batch, x, y)
        got = _c(y, batch, n)
        # the same passes, tables and geometry rules: identical bits
        assert np.array_equal(y.cpu().numpy(), ref.cpu().numpy()), f"n={n}: noalloc differs from tcfft_exec"
        check_rows(got, oracle.fft_batch(si.as_complex128(h)), PLAIN_TOL, f"noalloc n={n}")


@pytest.mark.parametrize("log2n,batch", [(21, 1), (22, 1), (23, 1), (24, 1), (23, 2), (16, 256)])
def test_noalloc_against_oracle(log2n, batch):
    # 2^22..2^24 run here as two passes (2048/4096-point strided and
    # contiguous passes) that no plan uses; n * batch = 2^24 is the limit
    import torch
    n = 1 << log2n
    h = si.half_input((batch, n), seed=80 + log2n)
    x = to_device(h)
    y = torch.full_like(x, 0x7E00)
    _noalloc(n, batch, x, y)
    check_rows(_c(y, batch, n), oracle.fft_batch(si.as_complex128(h)), PLAIN_TOL, f"noalloc 2^{log2n} x{batch}")


@pytest.mark.parametrize("log2n,batch", [(16, 3), (24, 1)])
def test_noalloc_in_place(log2n, batch):
    # in == out: pass 2 writes the buffer pass 1 read; the programmatic
    # dependent launch orders pass 2's reads of the workspace after pass 1
    n = 1 << log2n
    h = si.half_input((batch, n), seed=90 + log2n)
    x = to_device(h)
    _noalloc(n, batch, x, x)
    check_rows(_c(x, batch, n), oracle.fft_batch(si.as_complex128(h)), PLAIN_TOL, f"noalloc in place 2^{log2n}")


def test_noalloc_rejects_sizes_beyond_its_workspace():
    import torch
    import paper_2104_11471_gb300 as tc
    lib = tc.lib()
    x = torch.zeros(64, dtype=torch.uint16, device="cuda")
    p = ctypes.c_void_p(x.data_ptr())
    assert lib.tcfft_exec_1d_noalloc(ctypes.c_int64(1 << 24), ctypes.c_int64(2), p, p, None) == 1
    assert lib.tcfft_exec_1d_noalloc(ctypes.c_int64(1 << 14), ctypes.c_int64(1), p, p, None) == 1
    assert lib.tcfft_exec_1d_noalloc(ctypes.c_int64(3 << 15), ctypes.c_int64(1), p, p, None) == 1

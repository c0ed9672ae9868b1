"""The allocation-free entry point tcfft_exec_1d_noalloc against the plan path.

tcfft_exec_1d_noalloc serves callers that cannot allocate device memory when
they need a transform (a process that reserved its device-memory budget up
front, or a loop that must not pay for cudaMalloc/cudaFree).  It keeps its
workspace in a fixed device array shared by all calls, so this test runs two
different calls in a row and checks each against tcfft_plan_1d + tcfft_exec
on the same input.  This file is collected last on purpose; it must pass both
alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import seeded_inputs as si
from gpu_helpers import PLAIN_TOL, to_device

pytestmark = pytest.mark.gpu


def _run_plan(n, batch, x):
    import torch
    import paper_2104_11471_gb300 as tc
    y = torch.empty_like(x)
    plan = tc.Plan.plan_1d(n, batch)
    plan.exec(x, y)
    torch.cuda.synchronize()
    assert plan.last_error() == 0
    plan.destroy()
    return y


def test_noalloc_matches_plan_path_two_calls():
    import torch
    import oracle
    import paper_2104_11471_gb300 as tc
    lib = tc.lib()
    stream = torch.cuda.current_stream().cuda_stream
    for n, batch, seed in ((1 << 20, 3, 71), (1 << 16, 5, 72)):
        h = si.half_input((batch, n), seed=seed)
        x = to_device(h)
        ref = _run_plan(n, batch, x)
        y = torch.full_like(x, 0x7E00)
        st = lib.tcfft_exec_1d_noalloc(ctypes.c_int64(n), ctypes.c_int64(batch),
                                       ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                       ctypes.c_void_p(stream))
        assert st == 0, tc.STATUS.get(st)
        torch.cuda.synchronize()
        got = si.as_complex128(y.cpu().numpy().view(np.float16).reshape(batch, n, 2))
        want = si.as_complex128(ref.cpu().numpy().view(np.float16).reshape(batch, n, 2))
        assert np.all(np.isfinite(got))
        err = oracle.rel_l2_per_row(got, want)
        assert err.max() <= PLAIN_TOL, f"n={n}: rel-L2 to the plan path {err.max():.2e}"


def test_noalloc_rejects_sizes_beyond_its_workspace():
    import torch
    import paper_2104_11471_gb300 as tc
    lib = tc.lib()
    x = torch.zeros(64, dtype=torch.uint16, device="cuda")
    p = ctypes.c_void_p(x.data_ptr())
    assert lib.tcfft_exec_1d_noalloc(ctypes.c_int64(1 << 24), ctypes.c_int64(2), p, p, None) == 1
    assert lib.tcfft_exec_1d_noalloc(ctypes.c_int64(1 << 14), ctypes.c_int64(1), p, p, None) == 1
    assert lib.tcfft_exec_1d_noalloc(ctypes.c_int64(3 << 15), ctypes.c_int64(1), p, p, None) == 1

"""Failure detection without a GPU fault: the bounded device-side wait.

The kernel waits on a barrier that nothing completes; after the limit it must
report TCFFT_ERR_TIMEOUT and exit, leaving the context usable (a transform
runs correctly right after)."""
import numpy as np
import pytest

import oracle
from gpu_helpers import PLAIN_TOL, check_rows, fft1d_gpu

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives():
    import paper_2104_11471_gb300 as tc
    assert tc.lib().tcfft_selftest_wait_timeout(20_000_000) == 5  # ~10 ms at 2 GHz
    got, x = fft1d_gpu(1024, 4, seed=11)
    check_rows(got, oracle.fft_batch(x), PLAIN_TOL, "after timeout")


def test_invalid_arguments_on_gpu():
    import ctypes
    import torch
    import paper_2104_11471_gb300 as tc
    plan = tc.Plan.plan_1d(256, 4)
    x = torch.zeros(4 * 256 * 2 + 8, dtype=torch.float16, device="cuda")
    lib = tc.lib()
    # misaligned device pointers are rejected before any launch
    assert lib.tcfft_exec(plan.handle, ctypes.c_void_p(x.data_ptr() + 4), ctypes.c_void_p(x.data_ptr()),
                          None) == 2
    assert lib.tcfft_selftest_wait_timeout(-1) == 2
    plan.destroy()

"""tcfft_exec_host (host buffers, sliced upload / transform / download
pipeline for one-plane batches) against tcfft_exec on device buffers: the
same kernels per transform, so the results are equal bit for bit."""
import numpy as np
import pytest

import seeded_inputs as si

pytestmark = pytest.mark.gpu


def _both(plan, host_words):
    import torch
    hin = torch.from_numpy(np.ascontiguousarray(host_words).reshape(-1)).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    plan.exec_host(hin, hout)
    x = hin.to("cuda:0")
    y = torch.empty_like(x)
    plan.exec(x, y)
    torch.cuda.synchronize()
    assert plan.last_error() == 0
    return hout.numpy(), y.cpu().numpy()


@pytest.mark.parametrize("kind,shape,batch", [
    ("fp16", (4096,), 2048),        # single pass, sliced
    ("fp16", (1 << 16,), 128),      # two passes sharing the workspace, sliced
    ("fp16", (1 << 22,), 4),        # three passes, sliced
    ("fp16", (256, 256), 128),      # 2D, sliced
    ("fp32", (4096,), 1024),        # FP32 in/out, sliced
    ("split", (4096,), 1024),       # two planes: copy, run, copy back
    ("fp16", (256,), 8),            # small: copy, run, copy back
])
def test_exec_host_equals_exec(kind, shape, batch):
    import paper_2104_11471_gb300 as tc
    prec = {"fp16": tc.TCFFT_FP16, "split": tc.TCFFT_FP16_SPLIT, "fp32": tc.TCFFT_FP32}[kind]
    plan = (tc.Plan.plan_1d(shape[0], batch, prec) if len(shape) == 1
            else tc.Plan.plan_2d(shape[0], shape[1], batch, prec))
    try:
        full = (batch,) + tuple(shape)
        if kind == "fp32":
            words = si.float32_input(full, 41)
        elif kind == "split":
            hi, lo = si.split_input(full, 42)
            words = np.concatenate([hi.reshape(-1), lo.reshape(-1)]).view(np.uint16)
        else:
            words = si.half_input(full, 43).view(np.uint16)
        got_host, got_dev = _both(plan, words)
        assert got_host.nbytes == plan.io_bytes
        assert np.array_equal(got_host.view(np.uint8), got_dev.view(np.uint8))
    finally:
        plan.destroy()

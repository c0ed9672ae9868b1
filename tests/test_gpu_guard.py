"""Sanitizer substitute: guard bands around the caller's buffers.

Each plan runs with its input and output placed inside larger device
allocations whose bytes before and after are a canary pattern; after the
exec the canaries (and, out of place, the whole input) must be unchanged, so
no kernel writes outside the buffers it was given -- partial last chunks,
TMA boxes at the end of a tensor, ragged offset tables and sub-batch execs
included.  A plan that cannot get its workspace reports TCFFT_ERR_ALLOC."""
import numpy as np
import pytest

import seeded_inputs as si

pytestmark = pytest.mark.gpu

GUARD = 1 << 16  # bytes of canary on each side
CANARY = 0xA5


def _guarded(nbytes, fill=None):
    import torch
    buf = torch.full((GUARD + nbytes + GUARD,), CANARY, dtype=torch.uint8, device="cuda:0")
    if fill is not None:
        buf[GUARD:GUARD + nbytes] = torch.from_numpy(np.ascontiguousarray(fill).view(np.uint8).reshape(-1)).to("cuda:0")
    return buf


def _check(buf, nbytes, what):
    head = buf[:GUARD].cpu().numpy()
    tail = buf[GUARD + nbytes:].cpu().numpy()
    assert np.all(head == CANARY), f"{what}: write before the buffer"
    assert np.all(tail == CANARY), f"{what}: write after the buffer"


def _run(plan, words, batch=None):
    import torch
    nbytes = plan.io_bytes if batch is None else words.nbytes
    assert words.nbytes == nbytes
    xin = _guarded(nbytes, words)
    yout = _guarded(nbytes)
    x, y = xin[GUARD:GUARD + nbytes], yout[GUARD:GUARD + nbytes]
    if batch is None:
        plan.exec(x, y)
    else:
        plan.exec_batch(x, y, batch)
    torch.cuda.synchronize()
    assert plan.last_error() == 0
    _check(xin, nbytes, "input")
    _check(yout, nbytes, "output")
    assert np.array_equal(x.cpu().numpy(), np.ascontiguousarray(words).view(np.uint8).reshape(-1)), "input changed"
    return y


@pytest.mark.parametrize("kind,shape,batch,sub", [
    ("fp16", (4096,), 33, None),         # contiguous, TMA stores, partial last chunk
    ("fp16", (1024,), 3, None),          # leading radix 4, staging stores
    ("fp16", (1 << 16,), 5, None),       # two passes, TMA loads and stores
    ("fp16", (1 << 22,), 1, None),       # three passes
    ("fp16", (4096, 64), 3, None),       # 2D, two column passes
    ("fp16", (256, 256), 4, 3),          # 2D, sub-batch exec
    ("split", (1 << 16,), 3, None),      # split planes through the workspace
    ("fp32", (512, 512), 2, None),       # FP32 in/out
    ("fp32", (1 << 18,), 4, 3),          # FP32, sub-batch exec
])
def test_no_write_outside_the_buffers(kind, shape, batch, sub):
    import paper_2104_11471_gb300 as tc
    prec = {"fp16": tc.TCFFT_FP16, "split": tc.TCFFT_FP16_SPLIT, "fp32": tc.TCFFT_FP32}[kind]
    plan = (tc.Plan.plan_1d(shape[0], batch, prec) if len(shape) == 1
            else tc.Plan.plan_2d(shape[0], shape[1], batch, prec))
    try:
        n = sub or batch
        full = (n,) + tuple(shape)
        if kind == "fp32":
            words = si.float32_input(full, 7)
        elif kind == "split":
            hi, lo = si.split_input(full, 8)
            words = np.concatenate([hi.reshape(-1), lo.reshape(-1)]).view(np.uint16)
        else:
            words = si.half_input(full, 9).view(np.uint16)
        _run(plan, words, sub)
    finally:
        plan.destroy()


def test_ragged_no_write_outside_the_buffers():
    import paper_2104_11471_gb300 as tc
    shapes = [(256,), (1 << 15,), (64, 128), (4096,), (256,)]
    words = np.concatenate([si.half_input(s, 20 + i).reshape(-1, 2) for i, s in enumerate(shapes)]).view(np.uint16)
    plan = tc.Plan.plan_many(shapes, tc.TCFFT_FP16)
    try:
        _run(plan, words)
    finally:
        plan.destroy()


def test_workspace_allocation_failure_is_reported():
    # a 2^24-point transform batch whose workspace (4 TiB) no device has
    import paper_2104_11471_gb300 as tc
    with pytest.raises(tc.TcfftError) as e:
        tc.Plan.plan_1d(1 << 24, 1 << 16)
    assert e.value.status == 3  # TCFFT_ERR_ALLOC
    # the device stays usable
    plan = tc.Plan.plan_1d(256, 4)
    plan.destroy()

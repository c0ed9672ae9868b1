"""TCFFT_FP32: interleaved FP32 complex in and out, split-FP16 tensor-core
stages inside.  Every case against the FP64 oracle at the split-precision
bound (rel-L2 per transform), covering single-pass layouts (direct stores,
staging, leading radix), two- and three-pass 1D plans (FP16 hi / lo planes in
the workspace), 2D plans (FP32 between the row and column passes), ragged
batches, the inverse and exec_batch."""
import numpy as np
import pytest

import oracle
import seeded_inputs as si
from gpu_helpers import SPLIT_TOL, check_rows

pytestmark = pytest.mark.gpu


def _c128(f):
    f = np.asarray(f)
    return f[..., 0].astype(np.float64) + 1j * f[..., 1].astype(np.float64)


def _run(plan, x32, batch=None):
    import torch
    x = torch.from_numpy(np.ascontiguousarray(x32).reshape(-1)).to("cuda:0")
    y = torch.full_like(x, float("nan"))
    if batch is None:
        plan.exec(x, y)
    else:
        plan.exec_batch(x, y, batch)
    torch.cuda.synchronize()
    assert plan.last_error() == 0
    return y.cpu().numpy().reshape(x32.shape)


@pytest.mark.parametrize("log2n", [4, 8, 10, 11, 12, 13, 14, 15, 16, 18, 20])
def test_fp32_1d(log2n):
    import paper_2104_11471_gb300 as tc
    n = 1 << log2n
    batch = 3
    x = si.float32_input((batch, n), 300 + log2n)
    plan = tc.Plan.plan_1d(n, batch, tc.TCFFT_FP32)
    try:
        got = _c128(_run(plan, x))
    finally:
        plan.destroy()
    check_rows(got, oracle.fft_batch(_c128(x)), SPLIT_TOL, f"FP32 N=2^{log2n}")


def test_fp32_1d_three_pass():
    import paper_2104_11471_gb300 as tc
    n = 1 << 23
    x = si.float32_input((1, n), 323)
    plan = tc.Plan.plan_1d(n, 1, tc.TCFFT_FP32)
    try:
        assert plan.num_launches == 3
        got = _c128(_run(plan, x))
    finally:
        plan.destroy()
    check_rows(got, oracle.fft_batch(_c128(x)), SPLIT_TOL, "FP32 N=2^23")


@pytest.mark.parametrize("nx,ny,batch", [(16, 16, 2), (64, 128, 2), (256, 256, 1), (4096, 64, 1)])
def test_fp32_2d(nx, ny, batch):
    import paper_2104_11471_gb300 as tc
    x = si.float32_input((batch, nx, ny), nx + 7 * ny)
    plan = tc.Plan.plan_2d(nx, ny, batch, tc.TCFFT_FP32)
    try:
        got = _c128(_run(plan, x))
    finally:
        plan.destroy()
    ref = oracle.fft_2d(_c128(x))
    check_rows(got.reshape(batch, -1), ref.reshape(batch, -1), SPLIT_TOL, f"FP32 2D {nx}x{ny}")


def test_fp32_ragged():
    import paper_2104_11471_gb300 as tc
    shapes = [(256,), (1 << 15,), (64, 32), (256,), (4096,)]
    sizes = [int(np.prod(s)) for s in shapes]
    xs = [si.float32_input(s, 90 + i) for i, s in enumerate(shapes)]
    flat = np.concatenate([x.reshape(-1, 2) for x in xs])
    plan = tc.Plan.plan_many(shapes, tc.TCFFT_FP32)
    try:
        got = _c128(_run(plan, flat))
    finally:
        plan.destroy()
    off = 0
    for s, x, m in zip(shapes, xs, sizes):
        ref = oracle.fft_batch(_c128(x)[None]) if len(s) == 1 else oracle.fft_2d(_c128(x)[None])
        check_rows(got[off:off + m][None], ref.reshape(1, -1), SPLIT_TOL, f"FP32 ragged {s}")
        off += m


@pytest.mark.parametrize("n", [256, 4096, 1 << 16])
def test_fp32_round_trip(n):
    # forward, then inverse with 1/N: back to the input within the split bound
    import paper_2104_11471_gb300 as tc
    x = si.float32_input((2, n), 77)
    fwd = tc.Plan.plan_1d(n, 2, tc.TCFFT_FP32)
    inv = tc.Plan.plan_1d(n, 2, tc.TCFFT_FP32, tc.TCFFT_PLAN_INVERSE | tc.TCFFT_PLAN_SCALE)
    try:
        back = _c128(_run(inv, _run(fwd, x)))
    finally:
        fwd.destroy()
        inv.destroy()
    check_rows(back, _c128(x), 4 * SPLIT_TOL, f"FP32 round trip N={n}", c=2.0)


def test_fp32_exec_batch_prefix():
    import paper_2104_11471_gb300 as tc
    n = 1 << 15
    x = si.float32_input((5, n), 55)
    plan = tc.Plan.plan_1d(n, 8, tc.TCFFT_FP32)
    try:
        got = _c128(_run(plan, x, batch=5))
    finally:
        plan.destroy()
    check_rows(got, oracle.fft_batch(_c128(x)), SPLIT_TOL, "FP32 exec_batch")

"""Fused 2D passes: square matrices up to 512^2 (256^2 split) whose rows and
columns run in one launch, a cluster of CTAs per matrix exchanging the row
results through distributed shared memory (Sec. 3.1, 2D FFT).

The fused launch runs the same stage arithmetic as the two-pass plan (row
pass, FP16 intermediate, column pass), so its output must equal the two-pass
plan's bit for bit; both are checked against the FP64 oracle as well."""
import numpy as np
import pytest

import oracle
import seeded_inputs as si
from gpu_helpers import PLAIN_TOL, SPLIT_TOL, check_rows, run_plan

pytestmark = pytest.mark.gpu


def _plan(side, batch, split=False, flags=0, fused=True):
    import paper_2104_11471_gb300 as tc
    return tc.Plan.plan_2d(side, side, batch, tc.TCFFT_FP16_SPLIT if split else tc.TCFFT_FP16,
                           flags | (tc.TCFFT_PLAN_FUSED_2D if fused else 0))


def _planes(shape, seed, split):
    if split:
        hi, lo = si.split_input(shape, seed)
        return [hi, lo], si.split_value(hi, lo)
    h = si.half_input(shape, seed)
    return [h], si.as_complex128(h)


def _value(outs, split):
    return si.split_value(outs[0], outs[1]) if split else si.as_complex128(outs[0])


@pytest.mark.parametrize("side,batch,split", [(16, 3, False), (32, 5, False), (64, 2, False), (128, 3, False),
                                              (256, 2, False), (512, 2, False), (16, 2, True), (64, 3, True),
                                              (128, 2, True), (256, 2, True)])
def test_fused_equals_two_pass_and_oracle(side, batch, split):
    shape = (batch, side, side)
    planes, x = _planes(shape, side + batch, split)
    fused = _plan(side, batch, split)
    assert [d["mode"] for d in fused.describe()] == ["fused_2d"], fused.describe()
    got = run_plan(fused, planes, shape)
    fused.destroy()
    two = _plan(side, batch, split, fused=False)
    assert len(two.describe()) == 2
    ref_gpu = run_plan(two, planes, shape)
    two.destroy()
    for a, b in zip(got, ref_gpu):
        assert np.array_equal(a.view(np.uint16), b.view(np.uint16)), f"fused {side}^2 differs from the two-pass plan"
    ref = oracle.fft_2d(x)
    check_rows(_value(got, split).reshape(batch, -1), ref.reshape(batch, -1), SPLIT_TOL if split else PLAIN_TOL,
               f"fused 2D {side}^2 split={split}")


@pytest.mark.parametrize("side", [64, 256])
def test_fused_in_place_inverse_and_scale(side):
    import paper_2104_11471_gb300 as tc
    batch = 3
    shape = (batch, side, side)
    h = si.half_input(shape, 71)
    plan = _plan(side, batch, flags=tc.TCFFT_PLAN_INVERSE | tc.TCFFT_PLAN_SCALE)
    (o,) = run_plan(plan, [h], shape, inplace=True)
    plan.destroy()
    x = si.as_complex128(h)
    ref = np.conj(oracle.fft_2d(np.conj(x))) / (side * side)
    check_rows(si.as_complex128(o).reshape(batch, -1), ref.reshape(batch, -1), PLAIN_TOL, f"fused inverse {side}^2")


def test_fused_fp32_io():
    import torch
    import paper_2104_11471_gb300 as tc
    side, batch = 128, 2
    x = si.float32_input((batch, side, side), 72)
    plan = tc.Plan.plan_2d(side, side, batch, tc.TCFFT_FP32, tc.TCFFT_PLAN_FUSED_2D)
    assert plan.describe()[0]["mode"] == "fused_2d"
    xd = torch.from_numpy(x.reshape(-1)).cuda()
    y = torch.full_like(xd, float("nan"))
    plan.exec(xd, y)
    torch.cuda.synchronize()
    assert plan.last_error() == 0
    plan.destroy()
    g = y.cpu().numpy().reshape(batch, side, side, 2).astype(np.float64)
    got = g[..., 0] + 1j * g[..., 1]
    ref = oracle.fft_2d(x[..., 0].astype(np.float64) + 1j * x[..., 1].astype(np.float64))
    check_rows(got.reshape(batch, -1), ref.reshape(batch, -1), SPLIT_TOL, "fused FP32 128^2")


def test_fused_exec_batch_prefix_and_graph():
    import torch
    import paper_2104_11471_gb300 as tc
    from gpu_helpers import to_device
    side, batch = 256, 6
    h = si.half_input((batch, side, side), 73)
    x = to_device(h)
    plan = tc.Plan.plan_2d(side, side, batch, tc.TCFFT_FP16, tc.TCFFT_PLAN_GRAPH | tc.TCFFT_PLAN_FUSED_2D)
    y = torch.full_like(x, 0x7E00)
    plan.exec_batch(x, y, 2)  # the first two matrices only
    torch.cuda.synchronize()
    assert plan.last_error() == 0
    part = y.cpu().numpy().view(np.float16).reshape(batch, side, side, 2)
    assert np.all(np.isnan(part[2:].astype(np.float32)))  # untouched
    z = torch.full_like(x, 0x7E00)
    plan.exec(x, z)  # graph replay of the fused launch
    plan.exec(x, z)
    torch.cuda.synchronize()
    assert plan.last_error() == 0
    plan.destroy()
    full = z.cpu().numpy().view(np.float16).reshape(batch, side, side, 2)
    assert np.array_equal(full[:2].view(np.uint16), part[:2].view(np.uint16))
    ref = oracle.fft_2d(si.as_complex128(h))
    check_rows(si.as_complex128(full).reshape(batch, -1), ref.reshape(batch, -1), PLAIN_TOL, "fused graph 256^2")


def test_fused_ragged_square_groups():
    # ragged batch whose square 2D groups run fused (matrices at their own
    # offsets through the group's offset table) beside 1D groups
    import torch
    import paper_2104_11471_gb300 as tc
    from gpu_helpers import to_device
    shapes = [(64, 64), (1024,), (128, 128), (64, 64), (256, 256), (4096,), (128, 128), (32, 32)]
    pts = sum(int(np.prod(s)) for s in shapes)
    h = si.half_input((pts,), seed=74)
    plan = tc.Plan.plan_many(shapes, tc.TCFFT_FP16, tc.TCFFT_PLAN_GRAPH | tc.TCFFT_PLAN_FUSED_2D)
    assert any(d["mode"] == "fused_2d" for d in plan.describe())
    x = to_device(h)
    y = torch.full_like(x, 0x7E00)
    plan.exec(x, y)
    torch.cuda.synchronize()
    assert plan.last_error() == 0
    plan.destroy()
    out = si.as_complex128(y.cpu().numpy().view(np.float16).reshape(-1, 2))
    xin = si.as_complex128(h)
    off = 0
    for s in shapes:
        m = int(np.prod(s))
        ref = oracle.fft_batch(xin[off:off + m][None]) if len(s) == 1 else oracle.fft_2d(xin[off:off + m].reshape(s))
        check_rows(out[off:off + m][None], np.asarray(ref).reshape(1, -1), PLAIN_TOL, f"fused ragged {s}")
        off += m

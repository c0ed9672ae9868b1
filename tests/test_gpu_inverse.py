"""Inverse transform and 1/N scaling (plan flags), against the FP64 oracle
(inverse DFT = conj(DFT(conj(x)))) and as a forward -> inverse round trip."""
import numpy as np
import pytest

import oracle
import seeded_inputs as si
from gpu_helpers import PLAIN_TOL, SPLIT_TOL, U_PLAIN, U_SPLIT, check_elems, check_rows, run_plan, to_device

pytestmark = pytest.mark.gpu


def _plan(shape, batch, flags, split=False):
    import paper_2104_11471_gb300 as tc
    prec = tc.TCFFT_FP16_SPLIT if split else tc.TCFFT_FP16
    if len(shape) == 1:
        return tc.Plan.plan_1d(shape[0], batch, prec, flags)
    return tc.Plan.plan_2d(shape[0], shape[1], batch, prec, flags)


def _inv_ref(x, shape):
    f = oracle.fft_batch if len(shape) == 1 else oracle.fft_2d
    return np.conj(f(np.conj(x)))


@pytest.mark.parametrize("shape,batch", [((256,), 5), ((1024,), 3), ((4096,), 2), ((1 << 16,), 2),
                                         ((1 << 24,), 1), ((64, 128), 2), ((512, 512), 1)])
def test_inverse_matches_oracle(shape, batch):
    import paper_2104_11471_gb300 as tc
    h = si.half_input((batch,) + shape, seed=61)
    plan = _plan(shape, batch, tc.TCFFT_PLAN_INVERSE)
    (o,) = run_plan(plan, [h], (batch,) + shape)
    plan.destroy()
    x = si.as_complex128(h)
    check_rows(si.as_complex128(o).reshape(batch, -1), _inv_ref(x, shape).reshape(batch, -1), PLAIN_TOL,
               f"inverse {shape}")


@pytest.mark.parametrize("shape", [(256,), (1 << 20,), (256, 256)])
def test_round_trip_plain(shape):
    import torch
    import paper_2104_11471_gb300 as tc
    batch = 2
    h = si.half_input((batch,) + shape, seed=62)
    fwd = _plan(shape, batch, 0)
    inv = _plan(shape, batch, tc.TCFFT_PLAN_INVERSE | tc.TCFFT_PLAN_SCALE)
    x = to_device(h)
    y, z = torch.empty_like(x), torch.empty_like(x)
    fwd.exec(x, y)
    inv.exec(y, z)
    torch.cuda.synchronize()
    fwd.destroy()
    inv.destroy()
    back = si.as_complex128(z.cpu().numpy().view(np.float16).reshape((batch,) + shape + (2,)))
    assert oracle.rel_l2(back, si.as_complex128(h)) < 3e-3
    # two transforms' roundings: twice the per-element bound
    check_elems(back.reshape(batch, -1), si.as_complex128(h).reshape(batch, -1), U_PLAIN, f"round trip {shape}",
                c=2.0)


def test_round_trip_split_is_near_fp32():
    import torch
    import paper_2104_11471_gb300 as tc
    shape, batch = (4096,), 2
    hi, lo = si.split_input((batch,) + shape, seed=63)
    fwd = _plan(shape, batch, 0, split=True)
    inv = _plan(shape, batch, tc.TCFFT_PLAN_INVERSE | tc.TCFFT_PLAN_SCALE, split=True)
    x = to_device(np.concatenate([hi.reshape(-1), lo.reshape(-1)]))
    y, z = torch.empty_like(x), torch.empty_like(x)
    fwd.exec(x, y)
    inv.exec(y, z)
    torch.cuda.synchronize()
    fwd.destroy()
    inv.destroy()
    o = z.cpu().numpy().view(np.float16).reshape((2, batch) + shape + (2,))
    back, x = si.split_value(o[0], o[1]), si.split_value(hi, lo)
    assert oracle.rel_l2(back, x) < 4 * SPLIT_TOL
    check_elems(back, x, U_SPLIT, "split round trip", c=2.0)


def test_forward_scale_flag():
    import paper_2104_11471_gb300 as tc
    shape, batch = (1024,), 2
    h = si.half_input((batch,) + shape, seed=64)
    plan = _plan(shape, batch, tc.TCFFT_PLAN_SCALE)
    (o,) = run_plan(plan, [h], (batch,) + shape)
    plan.destroy()
    ref = oracle.fft_batch(si.as_complex128(h)) / 1024.0
    check_rows(si.as_complex128(o), ref, PLAIN_TOL, "scaled forward")

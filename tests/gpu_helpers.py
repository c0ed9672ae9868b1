"""Shared helpers for the GPU parity tests: run transforms through the C ABI
(python binding) on seeded inputs and return results beside the oracle's."""
from __future__ import annotations

import numpy as np

import oracle
import seeded_inputs as si

PLAIN_TOL = 5e-3   # rel-L2 bound for plain FP16 (per transform)
SPLIT_TOL = 2e-5   # rel-L2 bound for split FP16 (per transform)


def to_device(h: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(h).view(np.uint16).reshape(-1)).to("cuda:0")


def from_device(t, shape) -> np.ndarray:
    return t.cpu().numpy().view(np.float16).reshape(shape)


def run_plan(plan, planes: list[np.ndarray], shape, inplace: bool = False):
    """Copy the FP16 planes to the GPU, exec, return the output planes."""
    import torch
    x = to_device(np.concatenate([p.reshape(-1) for p in planes]))
    y = x if inplace else torch.full_like(x, 0x7E00)  # NaN fill: unwritten output shows up
    plan.exec(x, y)
    torch.cuda.synchronize()
    st = plan.last_error()
    assert st == 0, f"device status {st}"
    out = from_device(y, (len(planes),) + tuple(shape) + (2,))
    return [out[i] for i in range(len(planes))]


def fft1d_gpu(n: int, batch: int, seed: int, split: bool = False, inplace: bool = False):
    import paper_2104_11471_gb300 as tc
    prec = tc.TCFFT_FP16_SPLIT if split else tc.TCFFT_FP16
    plan = tc.Plan.plan_1d(n, batch, prec)
    try:
        if split:
            hi, lo = si.split_input((batch, n), seed)
            oh, ol = run_plan(plan, [hi, lo], (batch, n), inplace)
            return si.split_value(oh, ol), si.split_value(hi, lo)
        h = si.half_input((batch, n), seed)
        (o,) = run_plan(plan, [h], (batch, n), inplace)
        return si.as_complex128(o), si.as_complex128(h)
    finally:
        plan.destroy()


def fft2d_gpu(nx: int, ny: int, batch: int, seed: int, split: bool = False, inplace: bool = False):
    import paper_2104_11471_gb300 as tc
    prec = tc.TCFFT_FP16_SPLIT if split else tc.TCFFT_FP16
    plan = tc.Plan.plan_2d(nx, ny, batch, prec)
    try:
        shape = (batch, nx, ny)
        if split:
            hi, lo = si.split_input(shape, seed)
            oh, ol = run_plan(plan, [hi, lo], shape, inplace)
            return si.split_value(oh, ol), si.split_value(hi, lo)
        h = si.half_input(shape, seed)
        (o,) = run_plan(plan, [h], shape, inplace)
        return si.as_complex128(o), si.as_complex128(h)
    finally:
        plan.destroy()


def check_rows(got: np.ndarray, ref: np.ndarray, tol: float, what: str):
    assert np.all(np.isfinite(got)), f"{what}: non-finite output"
    errs = oracle.rel_l2_per_row(got, ref)
    assert errs.max() <= tol, f"{what}: max rel-L2 {errs.max():.3e} > {tol:.1e} (row {errs.argmax()})"
    return float(errs.max())

"""Shared helpers for the GPU parity tests: run transforms through the C ABI
(python binding) on seeded inputs and return results beside the oracle's.

Two bounds are checked for every transform:
  * rel-L2 per transform, ||X - X_ref||_2 / ||X_ref||_2 <= 5e-3 (plain FP16)
    or 2e-5 (split FP16 and FP32 I/O): the headline accuracy figure;
  * a per-element bound, for every output bin k of a length-N transform,
        |X[k] - X_ref[k]| <= c u log2(N) (||X_ref||_2 / sqrt(N) + |X_ref[k]|)
    with u = 2^-11 (FP16 storage, round to nearest) or 2^-22 (hi + 2^-11 lo
    pairs) and c = 1.  By Parseval ||X_ref||_2 / sqrt(N) is the input norm
    ||x||_2 (times the 1/N of a scaled transform), so the first term is the
    accumulated storage rounding of random data, the second the relative
    rounding of a bin that dominates (a tone).  The error model behind c: the
    per-bin error of random input is close to complex Gaussian with rms
    u sqrt(r/3) ||x||_2 over r roundings (r <= log16 N + 3, measured rel-L2
    0.7 u .. 1.3 u), whose maximum over 2^28 bins is below 4.4 rms, i.e.
    < 6 u ||x||_2 at N = 2^24 against a bound of 24 u ||x||_2.  One wrong bin
    moves rel-L2 by only about 1/sqrt(N), but it breaks this bound.
Structured inputs (deltas, tones) get one more term, c u log2(N) ||X_ref||_inf:
the rounding errors of periodic data are periodic too, so they do not spread
as white noise but gather in the few bins of the data's period (per-bin error
of order u |X_peak| / sqrt(period)).  Measured on the GPU over every plan
shape, plain and split: at most 0.26 u log2(N) ||X_ref||_inf off the peak.
"""
from __future__ import annotations

import math

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


U_PLAIN = 2.0 ** -11   # unit roundoff of FP16 storage
U_SPLIT = 2.0 ** -22   # hi + 2^-11 lo FP16 pairs


def unit_roundoff(tol: float) -> float:
    """u of the precision whose rel-L2 gate is `tol` (plain gates are >= 1e-3)."""
    return U_PLAIN if tol >= 1e-3 else U_SPLIT


def elem_bound(ref_rows: np.ndarray, u: float, c: float = 1.0, log2n: float | None = None,
               xnorm=None, coherent: bool = False) -> np.ndarray:
    """Per-element bound for rows of reference outputs (see the module text).

    ref_rows: [rows, bins] reference values.  log2n: log2 of the transform
    length (default: the row length); xnorm: per-row input norm times the
    transform's scale (default: ||X_ref||_2 / sqrt(N), exact for full rows);
    coherent: add the ||X_ref||_inf term of structured (periodic) inputs.
    """
    ref_rows = np.atleast_2d(np.asarray(ref_rows, dtype=np.complex128))
    n = ref_rows.shape[-1]
    lg = max(1.0, math.log2(n) if log2n is None else float(log2n))
    if xnorm is None:
        xnorm = np.linalg.norm(ref_rows, axis=1) / math.sqrt(n)
    xnorm = np.broadcast_to(np.asarray(xnorm, dtype=np.float64).reshape(-1), (ref_rows.shape[0],))
    mag = np.abs(ref_rows)
    scale = xnorm[:, None] + mag
    if coherent:
        scale = scale + mag.max(axis=1, keepdims=True)
    return c * u * lg * scale


def check_elems(got: np.ndarray, ref: np.ndarray, u: float, what: str, c: float = 1.0,
                log2n: float | None = None, xnorm=None, coherent: bool = False) -> float:
    """Every element within elem_bound; returns the worst error / bound ratio."""
    ref2 = np.atleast_2d(np.asarray(ref, dtype=np.complex128))
    got2 = np.asarray(got, dtype=np.complex128).reshape(ref2.shape)
    assert np.all(np.isfinite(got2)), f"{what}: non-finite output"
    bound = elem_bound(ref2, u, c, log2n, xnorm, coherent)
    ratio = np.abs(got2 - ref2) / bound
    worst = np.unravel_index(int(np.argmax(ratio)), ratio.shape)
    assert ratio[worst] <= 1.0, (f"{what}: element error {abs(got2[worst] - ref2[worst]):.3e} > bound "
                                 f"{bound[worst]:.3e} at row {worst[0]}, bin {worst[1]}")
    return float(ratio[worst])


def check_rows(got: np.ndarray, ref: np.ndarray, tol: float, what: str, c: float = 1.0,
               coherent: bool = False):
    """rel-L2 per transform <= tol and every element within the per-element bound."""
    assert np.all(np.isfinite(got)), f"{what}: non-finite output"
    errs = oracle.rel_l2_per_row(got, ref)
    assert errs.max() <= tol, f"{what}: max rel-L2 {errs.max():.3e} > {tol:.1e} (row {errs.argmax()})"
    ref2 = np.asarray(ref, dtype=np.complex128)
    ref2 = ref2.reshape(ref2.shape[0], -1) if ref2.ndim > 1 else ref2[None]
    check_elems(got, ref2, unit_roundoff(tol), what, c, coherent=coherent)
    return float(errs.max())

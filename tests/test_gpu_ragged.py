"""Ragged batches (tcfft_plan_many): mixed 1D lengths and 2D shapes in one
buffer, every transform checked against the FP64 oracle, and each result
identical alone and in the mix (graph replay and per-pass launches alike)."""
import numpy as np
import pytest

import oracle
import seeded_inputs as si
from gpu_helpers import PLAIN_TOL, SPLIT_TOL, check_rows, to_device

pytestmark = pytest.mark.gpu


def _shapes(seed, n1d, n2d, lo=4, hi=16, sides=(16, 32, 64, 128)):
    rng = np.random.default_rng(seed)
    shapes = [(1 << int(k),) for k in rng.integers(lo, hi + 1, size=n1d)]
    shapes += [(int(s), int(s)) for s in rng.choice(sides, size=n2d)]
    order = rng.permutation(len(shapes))
    return [shapes[i] for i in order]


def _run(shapes, planes, flags, split=False):
    import torch
    import paper_2104_11471_gb300 as tc
    prec = tc.TCFFT_FP16_SPLIT if split else tc.TCFFT_FP16
    plan = tc.Plan.plan_many(shapes, prec, flags)
    x = to_device(np.concatenate([p.reshape(-1) for p in planes]))
    y = torch.full_like(x, 0x7E00)
    plan.exec(x, y)
    plan.exec(x, y)  # a second replay of the same plan on the same buffers
    torch.cuda.synchronize()
    assert plan.last_error() == 0
    plan.destroy()
    return y.cpu().numpy().view(np.float16).reshape(len(planes), -1, 2)


def _check(got, ref, tol, s):
    """rel-L2 and the per-element bound of one transform of shape s."""
    check_rows(np.asarray(got).reshape(1, -1), np.asarray(ref).reshape(1, -1), tol, f"ragged {s}")


def _split_shapes(flat, shapes):
    out, off = [], 0
    for s in shapes:
        m = int(np.prod(s))
        out.append(flat[off:off + m].reshape(tuple(s) + flat.shape[1:]))
        off += m
    return out


@pytest.mark.parametrize("flags", [0, 2])
def test_ragged_mixed_plain_every_transform(flags):
    shapes = _shapes(3, 40, 8)
    pts = sum(int(np.prod(s)) for s in shapes)
    h = si.half_input((pts,), seed=31)
    out = _run(shapes, [h], flags)
    xs = _split_shapes(si.as_complex128(h), shapes)
    ys = _split_shapes(si.as_complex128(out[0]), shapes)
    for s, xin, got in zip(shapes, xs, ys):
        ref = oracle.fft_batch(xin) if len(s) == 1 else oracle.fft_2d(xin)
        _check(got, ref, PLAIN_TOL, s)


def test_ragged_split_precision():
    shapes = _shapes(4, 12, 3, lo=5, hi=13)
    pts = sum(int(np.prod(s)) for s in shapes)
    hi, lo = si.split_input((pts,), seed=32)
    out = _run(shapes, [hi, lo], 2, split=True)
    xs = _split_shapes(si.split_value(hi, lo), shapes)
    ys = _split_shapes(si.split_value(out[0], out[1]), shapes)
    for s, xin, got in zip(shapes, xs, ys):
        ref = oracle.fft_batch(xin) if len(s) == 1 else oracle.fft_2d(xin)
        _check(got, ref, SPLIT_TOL, s)


def test_ragged_two_pass_lengths():
    shapes = [(1 << 15,), (256,), (1 << 16,), (1 << 15,), (64, 64)]
    pts = sum(int(np.prod(s)) for s in shapes)
    h = si.half_input((pts,), seed=33)
    out = _run(shapes, [h], 2)
    for s, xin, got in zip(shapes, _split_shapes(si.as_complex128(h), shapes),
                           _split_shapes(si.as_complex128(out[0]), shapes)):
        ref = oracle.fft_batch(xin) if len(s) == 1 else oracle.fft_2d(xin)
        _check(got, ref, PLAIN_TOL, s)


def test_ragged_long_1d_groups():
    # the two-pass (four-step) groups of ragged plans from 2^17 to 2^24, one
    # transform each, mixed with a short transform and a small 2D shape
    shapes = [(1 << 20,), (1 << 17,), (1024,), (1 << 24,), (1 << 18,), (32, 64), (1 << 22,), (1 << 19,),
              (1 << 23,), (1 << 21,), (1 << 17,)]
    pts = sum(int(np.prod(s)) for s in shapes)
    h = si.half_input((pts,), seed=35)
    out = _run(shapes, [h], 2)
    for s, xin, got in zip(shapes, _split_shapes(si.as_complex128(h), shapes),
                           _split_shapes(si.as_complex128(out[0]), shapes)):
        ref = oracle.fft_batch(xin) if len(s) == 1 else oracle.fft_2d(xin)
        _check(got, ref, PLAIN_TOL, s)


def test_each_result_same_alone_and_in_mix():
    shapes = _shapes(5, 24, 4)
    pts = sum(int(np.prod(s)) for s in shapes)
    h = si.half_input((pts,), seed=34)
    mix = _run(shapes, [h], 2)[0]
    parts_in = _split_shapes(h.reshape(-1, 2), shapes)
    parts_mix = _split_shapes(mix, shapes)
    for i in (0, 7, len(shapes) - 1):
        alone = _run([shapes[i]], [parts_in[i]], 0)[0]
        assert np.array_equal(alone.reshape(-1, 2), parts_mix[i].reshape(-1, 2)), shapes[i]

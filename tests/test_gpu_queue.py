"""Persistent ragged executor (TCFFT_PLAN_PERSISTENT): every pass of a ragged
plan in one launch that claims (pass, chunk) items from a device work queue,
each pass waiting (bounded) for the previous pass of its group.

Each transform's arithmetic is the same as with one launch per pass, so the
results must equal the per-pass plan's bit for bit; they are checked against
the FP64 oracle as well.  The failure path runs a queue whose producer items
are withheld: the bounded wait must end with TCFFT_ERR_TIMEOUT, not a hang."""
import numpy as np
import pytest

import oracle
import seeded_inputs as si
from gpu_helpers import PLAIN_TOL, check_rows, to_device

pytestmark = pytest.mark.gpu


def _shapes():
    # single-pass and two-pass 1D lengths, square and rectangular 2D shapes
    # (lengths that both modes split alike: persistent plans run 1D lengths
    # above 8192 as two passes, per-pass plans only above 16384)
    return [(1 << 10,), (64, 64), (1 << 16,), (16,), (128, 256), (1 << 15,), (4096,), (256, 256), (1 << 20,),
            (1 << 13,), (32, 32), (1 << 16,), (512,), (1024, 128), (1 << 17,), (256,)]


def _check_all(shapes, h, got):
    xin, out = si.as_complex128(h), si.as_complex128(got)
    off = 0
    for s in shapes:
        m = int(np.prod(s))
        ref = oracle.fft_batch(xin[off:off + m][None]) if len(s) == 1 else oracle.fft_2d(xin[off:off + m].reshape(s))
        check_rows(out[off:off + m][None], np.asarray(ref).reshape(1, -1), PLAIN_TOL, f"persistent {s}")
        off += m


def _run(shapes, flags, h):
    import torch
    import paper_2104_11471_gb300 as tc
    plan = tc.Plan.plan_many(shapes, tc.TCFFT_FP16, flags)
    x = to_device(h)
    y = torch.full_like(x, 0x7E00)
    plan.exec(x, y)
    plan.exec(x, y)  # a second launch reuses the queue (counters reset per exec)
    torch.cuda.synchronize()
    assert plan.last_error() == 0
    desc, launches = plan.describe(), plan.num_launches
    plan.destroy()
    return y.cpu().numpy().view(np.float16).reshape(-1, 2), desc, launches


def test_persistent_equals_per_pass_and_oracle():
    import paper_2104_11471_gb300 as tc
    shapes = _shapes()
    pts = sum(int(np.prod(s)) for s in shapes)
    h = si.half_input((pts,), seed=91)
    got, desc, launches = _run(shapes, tc.TCFFT_PLAN_PERSISTENT, h)
    assert launches == 1 and all(d["queue"] == 1 for d in desc)
    ref_gpu, _, per_pass = _run(shapes, 0, h)
    assert per_pass > 1
    assert np.array_equal(got.view(np.uint16), ref_gpu.view(np.uint16)), "persistent launch differs from per-pass launches"
    _check_all(shapes, h, got)


def test_persistent_config_mix_against_oracle():
    # the ragged benchmark's kinds of shapes: 1D 2^8..2^16 (2^11 and 2^14 as
    # two passes here) and 2D sides 128..1024
    import paper_2104_11471_gb300 as tc
    shapes = [(1 << 14,), (128, 128), (1 << 8,), (1024, 1024), (1 << 16,), (512, 512), (1 << 11,), (1 << 14,),
              (256, 256), (1 << 9,), (1 << 11,)]
    pts = sum(int(np.prod(s)) for s in shapes)
    h = si.half_input((pts,), seed=94)
    got, desc, launches = _run(shapes, tc.TCFFT_PLAN_PERSISTENT, h)
    assert launches == 1
    _check_all(shapes, h, got)


def test_persistent_inverse_scaled_round_trip():
    import torch
    import paper_2104_11471_gb300 as tc
    shapes = [(1 << 16,), (256, 256), (2048,), (1 << 18,)]
    pts = sum(int(np.prod(s)) for s in shapes)
    h = si.half_input((pts,), seed=92)
    fwd = tc.Plan.plan_many(shapes, tc.TCFFT_FP16, tc.TCFFT_PLAN_PERSISTENT)
    inv = tc.Plan.plan_many(shapes, tc.TCFFT_FP16,
                            tc.TCFFT_PLAN_PERSISTENT | tc.TCFFT_PLAN_INVERSE | tc.TCFFT_PLAN_SCALE)
    x = to_device(h)
    y, z = torch.empty_like(x), torch.empty_like(x)
    fwd.exec(x, y)
    inv.exec(y, z)
    torch.cuda.synchronize()
    assert fwd.last_error() == 0 and inv.last_error() == 0
    fwd.destroy()
    inv.destroy()
    back = si.as_complex128(z.cpu().numpy().view(np.float16).reshape(-1, 2))
    xin = si.as_complex128(h)
    off = 0
    for s in shapes:
        m = int(np.prod(s))
        assert oracle.rel_l2(back[off:off + m], xin[off:off + m]) < 3e-3, s
        off += m


def test_withheld_dependency_times_out_and_context_survives():
    import paper_2104_11471_gb300 as tc
    from gpu_helpers import fft1d_gpu
    st = tc.lib().tcfft_selftest_queue_timeout(20_000_000)  # ~10 ms
    assert st == 5, tc.STATUS.get(st)  # TCFFT_ERR_TIMEOUT
    got, x = fft1d_gpu(4096, 3, seed=93)
    check_rows(got, oracle.fft_batch(x), PLAIN_TOL, "after queue timeout")

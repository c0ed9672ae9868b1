"""Structured inputs at every plan shape: deltas and tones, every output bin
against the FP64 oracle (Eq. dft_def).

A delta at n0 has X[k] = W_N^{n0 k} in every bin: magnitude one, its phase
stepping through the twiddle indices n0 k mod N.  A tone at k0 puts the whole
transform into bin k0.  Tones with one set bit in each base-16 digit position
(and in the leading radix-2/4/8 digit), plus k0 = N - 1 and N/2 + 1, pin the
output digit order of every pass bin by bin; deltas at 0, 1, N/2 + 1 and
N - 1 pin the twiddle indices.  A wrong digit permutation or twiddle index
moves a tone or rotates a delta's phase in exactly the bins it touches, which
the per-element bound catches where a rel-L2 gate could not (the bound here
carries the coherent ||X_ref||_inf term of periodic data).  The rows of one
batch are different structured inputs, rounded to FP16 (split: hi + lo
pairs); the oracle transforms exactly those values.
"""
import numpy as np
import pytest

import oracle
import seeded_inputs as si
from gpu_helpers import PLAIN_TOL, SPLIT_TOL, check_rows, run_plan

pytestmark = pytest.mark.gpu


def _rows_1d(n: int) -> list:
    lg = n.bit_length() - 1
    amp = min(0.5, 4096.0 / n)  # keeps the tone's bin N * amp inside FP16
    if lg <= 20:
        deltas = sorted({0, 1, n // 2 + 1, n - 1})
        bits = range(0, lg, 2)
    else:
        deltas = [1, n // 2 + 1]
        bits = range(1, lg, 4)
    tones = sorted({1 << b for b in bits} | {n - 1, n // 2 + 1})
    return [si.delta((n,), d) for d in deltas] + [si.tone(n, k, amp) for k in tones]


def _rows_2d(nx: int, ny: int) -> list:
    amp = min(0.5, 4096.0 / (nx * ny))
    lx, ly = nx.bit_length() - 1, ny.bit_length() - 1
    deltas = [(0, 0), (1, ny - 1), (nx // 2 + 1, 1), (nx - 1, ny // 2 + 1)]
    tones = [(1, 0), (0, 1), (nx - 1, ny - 1), (1 << (lx // 2), (1 << (ly // 2)) + 1), (nx // 2 + 1, 3 % ny),
             (1 << (lx - 1), 1 << (ly - 1))]
    return [si.delta((nx, ny), d) for d in deltas] + [si.tone_2d(nx, ny, a, b, amp) for a, b in tones]


def _run(shape, rows, split):
    import paper_2104_11471_gb300 as tc
    z = np.stack(rows)
    batch = z.shape[0]
    prec = tc.TCFFT_FP16_SPLIT if split else tc.TCFFT_FP16
    plan = (tc.Plan.plan_1d(shape[0], batch, prec) if len(shape) == 1
            else tc.Plan.plan_2d(shape[0], shape[1], batch, prec))
    try:
        if split:
            hi, lo = si.split_planes(z)
            oh, ol = run_plan(plan, [hi, lo], z.shape)
            return si.split_value(oh, ol), si.split_value(hi, lo)
        h = si.to_half_interleaved(z)
        (o,) = run_plan(plan, [h], z.shape)
        return si.as_complex128(o), si.as_complex128(h)
    finally:
        plan.destroy()


@pytest.mark.parametrize("log2n", list(range(4, 25)))
def test_structured_1d_plain(log2n):
    # single pass to 2^14, two passes 2^15..2^21, three passes 2^22..2^24
    n = 1 << log2n
    got, x = _run((n,), _rows_1d(n), False)
    check_rows(got, oracle.fft_batch(x), PLAIN_TOL, f"structured N=2^{log2n}", coherent=True)


@pytest.mark.parametrize("log2n", [4, 7, 8, 11, 12, 14, 15, 16, 19, 22, 23])
def test_structured_1d_split(log2n):
    n = 1 << log2n
    got, x = _run((n,), _rows_1d(n), True)
    check_rows(got, oracle.fft_batch(x), SPLIT_TOL, f"structured split N=2^{log2n}", coherent=True)


@pytest.mark.parametrize("nx,ny", [(16, 16), (128, 128), (256, 256), (512, 64), (64, 2048), (2048, 64),
                                   (1024, 1024), (4096, 32), (8192, 16)])
def test_structured_2d_plain(nx, ny):
    got, x = _run((nx, ny), _rows_2d(nx, ny), False)
    ref = oracle.fft_2d(x)
    b = got.shape[0]
    check_rows(got.reshape(b, -1), ref.reshape(b, -1), PLAIN_TOL, f"structured 2D {nx}x{ny}", coherent=True)


@pytest.mark.parametrize("nx,ny", [(16, 32), (256, 256), (2048, 64), (4096, 32)])
def test_structured_2d_split(nx, ny):
    got, x = _run((nx, ny), _rows_2d(nx, ny), True)
    ref = oracle.fft_2d(x)
    b = got.shape[0]
    check_rows(got.reshape(b, -1), ref.reshape(b, -1), SPLIT_TOL, f"structured split 2D {nx}x{ny}",
               coherent=True)

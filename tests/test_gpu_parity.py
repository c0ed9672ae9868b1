"""GPU parity: every result of the CUDA path against the FP64 oracle.

All transforms run through the C ABI (python binding) on seeded inputs
uniform in [-1, 1] (Sec. 5.1) rounded to FP16; the oracle transforms the
exact values the GPU received.  Bounds: rel-L2 per transform <= 5e-3
(plain FP16) and <= 2e-5 (split FP16), and every output element within the
per-element bound of gpu_helpers (c u log2 N (||x||_2 + |X_ref[k]|)).
"""
import numpy as np
import pytest

import oracle
import seeded_inputs as si
from gpu_helpers import PLAIN_TOL, SPLIT_TOL, check_elems, check_rows, fft1d_gpu, fft2d_gpu, unit_roundoff

pytestmark = pytest.mark.gpu


def test_smallest_config_n256_batch16():
    got, x = fft1d_gpu(256, 16, seed=0)
    ref = oracle.fft_batch(x)
    check_rows(got, ref, PLAIN_TOL, "N=256 batch=16")
    assert oracle.max_abs(got, ref) < 0.1


@pytest.mark.parametrize("log2n", list(range(4, 15)))
@pytest.mark.parametrize("batch", [1, 3, 33])
def test_1d_single_pass_sizes(log2n, batch):
    n = 1 << log2n
    got, x = fft1d_gpu(n, batch, seed=log2n * 100 + batch)
    check_rows(got, oracle.fft_batch(x), PLAIN_TOL, f"N={n} batch={batch}")


@pytest.mark.parametrize("log2n", [15, 16, 17, 18, 19, 20, 21])
def test_1d_two_pass_sizes(log2n):
    # the default plans: two passes from 2^15 up to 2^21 (2^21 = 2048 x 1024,
    # a 2048-point strided pass)
    n = 1 << log2n
    batch = 3
    got, x = fft1d_gpu(n, batch, seed=log2n)
    check_rows(got, oracle.fft_batch(x), PLAIN_TOL, f"N={n} batch={batch}")


@pytest.mark.parametrize("n,batch", [(256, 16), (4096, 5), (1 << 16, 2)])
def test_1d_in_place(n, batch):
    got, x = fft1d_gpu(n, batch, seed=7, inplace=True)
    check_rows(got, oracle.fft_batch(x), PLAIN_TOL, f"in-place N={n}")


@pytest.mark.parametrize("nx,ny,batch", [(16, 16, 2), (32, 64, 3), (64, 32, 1), (256, 256, 2),
                                         (128, 1024, 1), (1024, 128, 1), (512, 256, 2),
                                         (2048, 64, 2), (2048, 2048, 1), (4096, 32, 1), (8192, 16, 2)])
def test_2d_sizes(nx, ny, batch):
    got, x = fft2d_gpu(nx, ny, batch, seed=nx + ny)
    ref = oracle.fft_2d(x)
    check_rows(got.reshape(batch, -1), ref.reshape(batch, -1), PLAIN_TOL, f"2D {nx}x{ny}")


@pytest.mark.parametrize("log2n", [4, 8, 11, 12, 13, 14, 16])
def test_1d_split_precision(log2n):
    n = 1 << log2n
    got, x = fft1d_gpu(n, 3, seed=50 + log2n, split=True)
    check_rows(got, oracle.fft_batch(x), SPLIT_TOL, f"split N={n}")


@pytest.mark.parametrize("nx,ny", [(16, 32), (256, 256), (64, 1024), (2048, 64), (2048, 2048), (4096, 32)])
def test_2d_split_precision(nx, ny):
    # 2048 rows: one 2048-point strided column pass; 4096: two column passes
    got, x = fft2d_gpu(nx, ny, 2, seed=9, split=True)
    ref = oracle.fft_2d(x)
    check_rows(got.reshape(2, -1), ref.reshape(2, -1), SPLIT_TOL, f"split 2D {nx}x{ny}")


def test_deterministic_and_batch_independent():
    n = 4096
    a, x = fft1d_gpu(n, 9, seed=3)
    b, _ = fft1d_gpu(n, 9, seed=3)
    assert np.array_equal(a, b)
    # the same transform alone gives bit-identical output
    import paper_2104_11471_gb300 as tc
    from gpu_helpers import run_plan
    h = si.half_input((9, n), seed=3)
    plan = tc.Plan.plan_1d(n, 1)
    (o,) = run_plan(plan, [h[4:5]], (1, n))
    plan.destroy()
    assert np.array_equal(si.as_complex128(o)[0], a[4])


# --------------------------------------------------------------- full sizes
def _full_size_rows(shape, batch, seed, split, rows):
    """Run one plan at a benchmark size; return sampled transforms and their inputs."""
    import torch
    import paper_2104_11471_gb300 as tc
    from gpu_helpers import to_device
    prec = tc.TCFFT_FP16_SPLIT if split else tc.TCFFT_FP16
    plan = (tc.Plan.plan_1d(shape[0], batch, prec) if len(shape) == 1
            else tc.Plan.plan_2d(shape[0], shape[1], batch, prec))
    pts = int(np.prod(shape))
    try:
        rng = np.random.default_rng(seed)
        if split:
            hi, lo = si.split_input((batch,) + tuple(shape), seed)
            x = to_device(np.concatenate([hi.reshape(-1), lo.reshape(-1)]))
        else:
            h = si.half_input((batch,) + tuple(shape), seed)
            x = to_device(h)
        y = torch.full_like(x, 0x7E00)
        plan.exec(x, y)
        torch.cuda.synchronize()
        assert plan.last_error() == 0
        pick = sorted(set([0, batch - 1] + list(rng.integers(0, batch, size=rows))))
        planes = 2 if split else 1
        yv = y.view(planes, batch, pts * 2)
        out = []
        for b in pick:
            o = yv[:, b].cpu().numpy().view(np.float16).reshape((planes,) + tuple(shape) + (2,))
            if split:
                got = si.split_value(o[0], o[1])
                xin = si.split_value(hi[b], lo[b])
            else:
                got = si.as_complex128(o[0])
                xin = si.as_complex128(h[b])
            out.append((got, xin))
        return out
    finally:
        plan.destroy()


@pytest.mark.parametrize("log2n", [8, 10, 12, 14, 16, 18, 20, 22, 24])
def test_1d_sweep_full_size_sampled(log2n):
    # the benchmark's configuration: 2^28 points per exec, batch = 2^28 / N
    n = 1 << log2n
    batch = (1 << 28) // n
    for got, xin in _full_size_rows((n,), batch, si.sweep_seed(log2n), False, rows=2):
        ref = oracle.fft_batch(xin[None, :])[0]
        check_rows(got[None], ref[None], PLAIN_TOL, f"N=2^{log2n}")


@pytest.mark.parametrize("side,split", [(256, False), (512, False), (1024, False), (4096, False),
                                        (8192, False), (256, True), (1024, True), (4096, True),
                                        (8192, True)])
def test_2d_full_size_sampled(side, split):
    batch = (1 << 28) // (side * side)
    tol = SPLIT_TOL if split else PLAIN_TOL
    lg = side.bit_length() - 1
    for got, xin in _full_size_rows((side, side), batch, si.seed_2d(lg), split, rows=1):
        ref = oracle.fft_2d(xin)
        check_rows(got.reshape(1, -1), ref.reshape(1, -1), tol, f"2D {side}^2 split={split}")


def test_max_abs_within_fp16_range_at_2e24():
    # the largest 1D outputs must stay finite in FP16 (no hidden scaling)
    n = 1 << 24
    for got, xin in _full_size_rows((n,), 16, 7, False, rows=0):
        assert np.max(np.abs(got)) < 65504


def test_plans_sharing_a_kernel_with_different_shared_memory():
    # two plans whose passes use the same kernel with different shared-memory
    # sizes: creating the second must not break launches of the first
    import torch
    import paper_2104_11471_gb300 as tc
    from gpu_helpers import run_plan
    big = tc.Plan.plan_1d(16, 1024)          # contiguous, 512 transforms per CTA
    small = tc.Plan.plan_2d(16, 16, 3)       # same length, small row/column blocks
    h = si.half_input((1024, 16), seed=5)
    (o,) = run_plan(big, [h], (1024, 16))
    check_rows(si.as_complex128(o), oracle.fft_batch(si.as_complex128(h)), PLAIN_TOL, "after second plan")
    big.destroy()
    small.destroy()


@pytest.mark.parametrize("log2n,batch", [(24, 1), (22, 2), (21, 3)])
def test_1d_three_pass_split(log2n, batch, monkeypatch):
    # the three-pass decomposition (forced down to 2^21 here) against the oracle
    monkeypatch.setenv("TCFFT_THREE_PASS_MIN", "21")
    n = 1 << log2n
    got, x = fft1d_gpu(n, batch, seed=log2n + 40)
    check_rows(got, oracle.fft_batch(x), PLAIN_TOL, f"three-pass N=2^{log2n}")


@pytest.mark.parametrize("log2n,batch,split", [(25, 2, False), (26, 1, False), (27, 1, False),
                                               (23, 1, True), (25, 1, True)])
def test_1d_beyond_2e24_sampled_bins(log2n, batch, split):
    # three-pass plans past the benchmark sweep (and split precision past
    # 2^22): sampled output bins of the first and last transform against
    # direct FP64 sums (rel-L2 over the bins)
    n = 1 << log2n
    tol = SPLIT_TOL if split else PLAIN_TOL
    rng = np.random.default_rng(log2n)
    bins = np.unique(np.concatenate([[0, 1, n // 2, n - 1], rng.integers(0, n, size=28)]))
    for got, xin in _full_size_rows((n,), batch, 60 + log2n, split, rows=0):
        assert np.all(np.isfinite(got))
        ref = oracle.dft_bins(xin, bins)
        err = oracle.rel_l2(got[bins], ref)
        assert err <= tol, f"N=2^{log2n} split={split}: sampled rel-L2 {err:.2e}"
        check_elems(got[bins], ref, unit_roundoff(tol), f"N=2^{log2n} sampled bins", log2n=log2n,
                    xnorm=np.linalg.norm(xin))

"""Pins for the FP64 CPU oracle (CPU only).

The oracle is the reference every GPU result is compared against, so it is
pinned here to things other than itself: hand-worked DFTs (tests/golden),
closed forms, Parseval, linearity, the inverse round trip, the shift theorem,
brute force on small sizes, 2D separability and numpy's pocketfft.  The
mutation tests at the end compile the oracle with planted mistakes and check
that these pins catch each one.
"""
import math
import os

import numpy as np
import pytest

import oracle
import seeded_inputs as si


def _parse_golden(path):
    cases = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, n, xs, Xs = [p.strip() for p in line.split("|")]

            def cplx_list(s):
                return np.array([complex(float(a), float(b))
                                 for a, b in (t.split(",") for t in s.split(";"))])
            cases.append((name, int(n), cplx_list(xs), cplx_list(Xs)))
    return cases


def test_golden_hand_examples(golden_dir):
    cases = _parse_golden(os.path.join(golden_dir, "dft_hand_examples.txt"))
    assert len(cases) >= 5
    for name, n, x, X in cases:
        assert x.shape == (n,) and X.shape == (n,), name
        for fn in (oracle.dft_brute, oracle.fft_radix2):
            got = fn(x)
            np.testing.assert_allclose(got, X, rtol=0, atol=1e-13, err_msg=name)


# ------------------------------------------------------------------ twiddles
def test_twiddle_special_angles():
    s = math.sqrt(0.5)
    expect = {(0, 8): 1, (1, 8): complex(s, -s), (2, 8): -1j, (3, 8): complex(-s, -s),
              (4, 8): -1, (5, 8): complex(-s, s), (6, 8): 1j, (7, 8): complex(s, s),
              (1, 4): -1j, (1, 2): -1, (3, 4): 1j, (1, 12): complex(math.sqrt(3) / 2, -0.5)}
    for (a, n), w in expect.items():
        assert abs(oracle.twiddle(a, n) - w) < 2e-16, (a, n)


def test_twiddle_periodic_and_unit():
    for n in (16, 1 << 12, 1 << 24, 1 << 27):
        for a in (1, 3, n // 8 + 1, n // 3, n - 1, 5 * n + 7, -3):
            w = oracle.twiddle(a, n)
            assert abs(abs(w) - 1.0) < 4e-16
            assert abs(w - oracle.twiddle(a % n, n)) == 0.0


def test_twiddle_matches_complex_exp():
    rng = np.random.default_rng(7)
    for n in (1 << 5, 1 << 13, 1 << 24):
        for a in rng.integers(0, n, size=64):
            ref = np.exp(-2j * np.pi * (int(a) / n))
            assert abs(oracle.twiddle(int(a), n) - ref) < 1e-15


def test_twiddle_group_law():
    n = 1 << 20
    rng = np.random.default_rng(3)
    for a, b in rng.integers(0, n, size=(50, 2)):
        lhs = oracle.twiddle(int(a), n) * oracle.twiddle(int(b), n)
        assert abs(lhs - oracle.twiddle(int(a + b), n)) < 1e-15


# ------------------------------------------------------------- closed forms
@pytest.mark.parametrize("fn", ["dft_brute", "fft_radix2"])
@pytest.mark.parametrize("n", [1, 2, 4, 16, 64])
def test_closed_forms(fn, n):
    f = getattr(oracle, fn)
    delta = np.zeros(n, complex)
    delta[0] = 1
    np.testing.assert_allclose(f(delta), np.ones(n), atol=1e-14)
    c = 0.3 - 0.7j
    X = f(np.full(n, c))
    expect = np.zeros(n, complex)
    expect[0] = c * n
    np.testing.assert_allclose(X, expect, atol=1e-13 * n)
    for k0 in sorted({0, 1 % n, n // 2, n - 1}):
        tone = np.exp(2j * np.pi * k0 * np.arange(n) / n)
        expect = np.zeros(n, complex)
        expect[k0] = n
        np.testing.assert_allclose(f(tone), expect, atol=1e-12 * n)


def test_delayed_delta():
    n = 32
    for n0 in (1, 5, 31):
        x = np.zeros(n, complex)
        x[n0] = 1
        expect = np.array([oracle.twiddle(n0 * k, n) for k in range(n)])
        np.testing.assert_allclose(oracle.fft_radix2(x), expect, atol=1e-15)
        np.testing.assert_allclose(oracle.dft_brute(x), expect, atol=1e-15)


# ---------------------------------------------------------- brute force pins
@pytest.mark.parametrize("n", [2, 4, 8, 16, 32, 64])
def test_radix2_matches_brute(n):
    x = si.uniform_complex((n,), seed=n)
    np.testing.assert_allclose(oracle.fft_radix2(x), oracle.dft_brute(x), atol=1e-13)


@pytest.mark.parametrize("n,radices", [
    (16, [16]), (16, [4, 4]), (16, [2, 8]), (32, [2, 16]), (32, [16, 2]),
    (64, [4, 16]), (64, [16, 4]), (64, [2, 2, 2, 2, 2, 2]), (128, [8, 16]),
    (256, [16, 16]), (512, [2, 16, 16]), (512, [16, 16, 2]), (1024, [4, 16, 16]),
    (4096, [16, 16, 16]), (8192, [8, 16, 16, 4]),
])
def test_mixed_matches_radix2_and_brute(n, radices):
    x = si.uniform_complex((n,), seed=100 + n)
    ref = oracle.fft_radix2(x)
    got = oracle.fft_mixed(x, radices)
    np.testing.assert_allclose(got, ref, atol=1e-12 * math.sqrt(n))
    if n <= 64:
        np.testing.assert_allclose(got, oracle.dft_brute(x), atol=1e-13)


def test_mixed_rejects_bad_radices():
    with pytest.raises(ValueError):
        oracle.fft_mixed(np.zeros(16, complex), [4, 8])


def test_merge_is_one_cooley_tukey_step():
    # X_in rows are the DFTs of x_m[n] = x[n N1 + m]; one merge gives the full DFT.
    for n1, n2 in ((16, 16), (16, 4), (2, 32), (4, 16), (16, 1)):
        n = n1 * n2
        x = si.uniform_complex((n,), seed=n1 * 1000 + n2)
        xin = np.stack([oracle.dft_brute(x[m::n1]) for m in range(n1)])
        xout = oracle.merge(xin)
        np.testing.assert_allclose(xout.reshape(-1), oracle.dft_brute(x), atol=1e-12)


def test_dft_bins_matches_brute():
    n = 512
    x = si.uniform_complex((n,), seed=5)
    bins = np.array([0, 1, 7, 255, 256, 511, 1023])
    got = oracle.dft_bins(x, bins, nthreads=3)
    ref = oracle.dft_brute(x)[bins % n]
    np.testing.assert_allclose(got, ref, atol=1e-12)


# --------------------------------------------------------------- invariants
@pytest.mark.parametrize("n", [256, 4096, 1 << 16])
def test_parseval_linearity_inverse_shift(n):
    x = si.uniform_complex((n,), seed=11)
    y = si.uniform_complex((n,), seed=12)
    X = oracle.fft_radix2(x)
    Y = oracle.fft_radix2(y)
    # Parseval
    assert abs(np.sum(abs(X) ** 2) - n * np.sum(abs(x) ** 2)) < 1e-11 * n * np.sum(abs(x) ** 2)
    # linearity
    a, b = 0.7 - 0.2j, -1.3 + 0.5j
    np.testing.assert_allclose(oracle.fft_radix2(a * x + b * y), a * X + b * Y,
                               atol=1e-12 * math.sqrt(n))
    # inverse round trip: conj(FFT(conj(X))) / n = x
    back = np.conj(oracle.fft_radix2(np.conj(X))) / n
    np.testing.assert_allclose(back, x, atol=1e-13)
    # circular shift by s multiplies X[k] by W_n^{s k}
    s = 3
    Xs = oracle.fft_radix2(np.roll(x, s))
    ramp = np.array([oracle.twiddle(s * k, n) for k in range(n)])
    np.testing.assert_allclose(Xs, X * ramp, atol=1e-11 * math.sqrt(n))


def test_real_input_hermitian():
    n = 1024
    x = si.uniform_complex((n,), seed=4).real.astype(complex)
    X = oracle.fft_radix2(x)
    np.testing.assert_allclose(X[1:], np.conj(X[1:][::-1]), atol=1e-12)


@pytest.mark.parametrize("n", [16, 256, 1024, 1 << 14, 1 << 18])
def test_matches_numpy_pocketfft(n):
    x = si.uniform_complex((4, n), seed=n)
    got = oracle.fft_batch(x, nthreads=4)
    ref = np.fft.fft(x, axis=-1)
    assert oracle.rel_l2(got, ref) < 1e-14


# ------------------------------------------------------------------- 2D
@pytest.mark.parametrize("nx,ny", [(16, 16), (32, 64), (128, 16), (256, 256)])
def test_2d_separable_and_numpy(nx, ny):
    x = si.uniform_complex((3, nx, ny), seed=nx + ny)
    got = oracle.fft_2d(x, nthreads=4)
    rows = oracle.fft_batch(x.reshape(-1, ny)).reshape(3, nx, ny)
    cols = oracle.fft_batch(np.swapaxes(rows, 1, 2).reshape(-1, nx))
    sep = np.swapaxes(cols.reshape(3, ny, nx), 1, 2)
    np.testing.assert_allclose(got, sep, atol=1e-12 * math.sqrt(nx * ny))
    assert oracle.rel_l2(got, np.fft.fft2(x)) < 1e-14


def test_2d_brute_small():
    nx, ny = 4, 8
    x = si.uniform_complex((nx, ny), seed=9)
    X = oracle.fft_2d(x)
    for k1 in range(nx):
        for k2 in range(ny):
            ref = sum(x[a, b] * oracle.twiddle(a * k1, nx) * oracle.twiddle(b * k2, ny)
                      for a in range(nx) for b in range(ny))
            assert abs(X[k1, k2] - ref) < 1e-13


# ------------------------------------------------------------------ metrics
def test_metrics():
    ref = np.array([3 + 4j, 0, 1j])
    got = ref + np.array([0.03 + 0.04j, 0, 0])
    assert abs(oracle.rel_l2(got, ref) - 0.05 / math.sqrt(26)) < 1e-15
    assert abs(oracle.max_abs(got, ref) - 0.05) < 1e-15
    # bin 1 (|ref| = 0) is skipped; mean over the other two = (0.01 + 0) / 2
    assert abs(oracle.mean_rel_err(got, ref) - 0.005) < 1e-15


# ------------------------------------------------------- seeded inputs
def test_seeded_inputs_are_fp16_and_reproducible():
    h = si.half_input((8, 64), seed=0)
    assert h.dtype == np.float16 and h.shape == (8, 64, 2)
    assert np.array_equal(h, si.half_input((8, 64), seed=0))
    assert np.all(np.abs(h.astype(np.float64)) <= 1.0)
    z = si.uniform_complex((1000,), seed=1)
    hi, lo = si.split_planes(z)
    # the split pair carries ~22 significant bits
    err = np.abs(si.split_value(hi, lo) - z)
    assert np.max(err / np.maximum(np.abs(z), 1e-3)) < 2.0 ** -20


# ------------------------------------------------------------ mutation pins
def _pins_catch(v):
    """Run a subset of the pins against an oracle variant; True if any fails."""
    failures = 0
    x = si.uniform_complex((64,), seed=1)
    try:
        np.testing.assert_allclose(v.fft_radix2(x), np.fft.fft(x), atol=1e-12)
    except AssertionError:
        failures += 1
    try:
        np.testing.assert_allclose(v.dft_brute(x), np.fft.fft(x), atol=1e-12)
    except AssertionError:
        failures += 1
    try:
        np.testing.assert_allclose(v.fft_mixed(x, [4, 16]), np.fft.fft(x), atol=1e-12)
    except AssertionError:
        failures += 1
    x2 = si.uniform_complex((2, 8, 16), seed=2)
    try:
        np.testing.assert_allclose(v.fft_2d(x2, nthreads=1), np.fft.fft2(x2), atol=1e-12)
    except AssertionError:
        failures += 1
    return failures


@pytest.mark.parametrize("plant", [1, 2, 3, 4, 5, 6])
def test_planted_mistakes_are_caught(plant, tmp_path):
    v = oracle.planted_variant(plant, str(tmp_path))
    assert _pins_catch(v) > 0


def test_unplanted_oracle_passes_mutation_pins():
    assert _pins_catch(oracle) == 0

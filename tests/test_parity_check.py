"""The parity checker itself (CPU only): the per-element bound used by every
GPU parity test must accept the FP16 storage rounding the method makes and
reject a result with one thin slice of wrong output bins.

Both sides are produced by the FP64 oracle on the CPU: the "wrong" result is
the oracle compiled with a planted mistake (a twiddle index taken N/8 too far
for the bins k = 3 mod N/16 in the last radix-2 merge, Eq. dft_s2), the
"right" one by the oracle as it stands plus FP16-sized noise.
"""
import numpy as np
import pytest

import oracle
import seeded_inputs as si
from gpu_helpers import PLAIN_TOL, U_PLAIN, U_SPLIT, check_elems, check_rows, elem_bound


def _fp16_roundings(z: np.ndarray, times: int, seed: int) -> np.ndarray:
    """z with `times` rounds of relative FP16-sized noise (u = 2^-11 per component)."""
    rng = np.random.default_rng(seed)
    out = z.copy()
    for _ in range(times):
        out = out.real * (1 + U_PLAIN * rng.uniform(-1, 1, z.shape)) + \
            1j * out.imag * (1 + U_PLAIN * rng.uniform(-1, 1, z.shape))
    return out


def test_planted_thin_slice_passes_rel_l2_but_fails_elementwise(tmp_path):
    n = 1 << 20
    x = si.as_complex128(si.half_input((1, n), seed=11))
    good = oracle.fft_batch(x)
    bad = oracle.planted_variant(6, str(tmp_path)).fft_batch(x)
    wrong = np.flatnonzero(np.abs(bad - good)[0] > 1e-6)
    assert 0 < wrong.size <= 16, wrong.size  # only the planted slice differs
    # the norm gate alone does not see it ...
    assert oracle.rel_l2_per_row(bad, good).max() < PLAIN_TOL
    # ... the per-element bound does
    with pytest.raises(AssertionError, match="element error"):
        check_elems(bad, good, U_PLAIN, "planted slice")
    with pytest.raises(AssertionError):
        check_rows(bad, good, PLAIN_TOL, "planted slice")


@pytest.mark.parametrize("log2n", [4, 8, 16])
def test_bound_accepts_fp16_storage_rounding(log2n):
    # rounding noise of one FP16 store per radix-16 stage plus input and output
    n = 1 << log2n
    x = si.uniform_complex((4, n), seed=log2n)
    ref = oracle.fft_batch(x)
    stages = log2n // 4 + 2
    noisy = oracle.fft_batch(_fp16_roundings(x, stages, seed=1))
    noisy = _fp16_roundings(noisy, 1, seed=2)
    ratio = check_elems(noisy, ref, U_PLAIN, f"noisy N={n}")
    assert ratio < 0.5


def test_bound_of_a_tone_follows_its_large_bin():
    # a tone concentrates the output in one bin: its relative rounding is
    # covered by the |X_ref[k]| term, the other bins by the input-norm term
    n = 4096
    k0 = 37
    t = np.exp(2j * np.pi * k0 * np.arange(n) / n) / 8
    ref = oracle.fft_batch(t[None])
    b = elem_bound(ref, U_PLAIN)
    assert np.isclose(abs(ref[0, k0]), n / 8)
    assert b[0, k0] > 12 * U_PLAIN * (n / 8)
    assert np.all(b[0, np.arange(n) != k0] < b[0, k0] / 10)


def test_split_bound_is_tighter_than_plain():
    ref = oracle.fft_batch(si.uniform_complex((2, 1024), seed=3))
    assert elem_bound(ref, U_SPLIT) * 2 ** 11 == pytest.approx(elem_bound(ref, U_PLAIN))

"""Seeded synthetic inputs shared by the oracle-side and GPU-side tests.

This module holds no FFT arithmetic.  It only draws numbers: the paper's
workloads are random sequences uniform in [-1, 1] (Sec. 5.1, "TestCase"), and
every draw here is seeded so both sides see the same values.

Complex values are returned in two forms:
  * ``half_interleaved`` -- numpy float16 array [..., n, 2] (re, im), the
    exact bytes the GPU library receives (interleaved FP16 complex);
  * ``as_complex128``    -- the same FP16 values widened exactly to FP64.
For the split-precision form a value v is stored as hi = fp16(v) and
lo = fp16((v - hi) * 2^11), two planes of the same shape.
"""
from __future__ import annotations

import numpy as np

SPLIT_SCALE = 2048.0  # lo plane carries (v - hi) * 2^11


def uniform_complex(shape, seed: int) -> np.ndarray:
    """FP64 complex draw, re and im i.i.d. uniform[-1, 1]."""
    rng = np.random.default_rng(seed)
    re = rng.uniform(-1.0, 1.0, size=shape)
    im = rng.uniform(-1.0, 1.0, size=shape)
    return re + 1j * im


def to_half_interleaved(z: np.ndarray) -> np.ndarray:
    """Round a complex array to FP16 (round to nearest even), [..., 2]."""
    out = np.empty(z.shape + (2,), dtype=np.float16)
    out[..., 0] = z.real.astype(np.float16)
    out[..., 1] = z.imag.astype(np.float16)
    return out


def as_complex128(h: np.ndarray) -> np.ndarray:
    """Widen an interleaved FP16 array [..., 2] exactly to complex128."""
    h = np.asarray(h)
    return h[..., 0].astype(np.float64) + 1j * h[..., 1].astype(np.float64)


def half_input(shape, seed: int) -> np.ndarray:
    """The plain-precision input: FP16 interleaved complex of `shape`."""
    return to_half_interleaved(uniform_complex(shape, seed))


def split_planes(z: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Split a complex FP64 array into (hi, lo) FP16 interleaved planes."""
    hi = to_half_interleaved(z)
    hi_c = as_complex128(hi)
    lo = to_half_interleaved((z - hi_c) * SPLIT_SCALE)
    return hi, lo


def split_value(hi: np.ndarray, lo: np.ndarray) -> np.ndarray:
    """The FP64 value a (hi, lo) pair represents: hi + lo * 2^-11."""
    return as_complex128(hi) + as_complex128(lo) / SPLIT_SCALE


def split_input(shape, seed: int) -> tuple[np.ndarray, np.ndarray]:
    return split_planes(uniform_complex(shape, seed))


def float32_input(shape, seed: int) -> np.ndarray:
    """The FP32-precision input: interleaved FP32 complex [..., 2] (round to nearest)."""
    z = uniform_complex(shape, seed)
    out = np.empty(z.shape + (2,), dtype=np.float32)
    out[..., 0] = z.real.astype(np.float32)
    out[..., 1] = z.imag.astype(np.float32)
    return out


def sweep_seed(log2n: int) -> int:
    """Seed of the 1D sweep at N = 2^log2n."""
    return 1000 + log2n


def seed_2d(log2side: int) -> int:
    return 2000 + log2side


# ------------------------------------------------------- structured inputs
def delta(shape, pos) -> np.ndarray:
    """FP64 complex array of `shape` with a single 1 at index `pos` (a tuple
    for 2D shapes), zero elsewhere."""
    z = np.zeros(shape, dtype=np.complex128)
    z[pos] = 1.0
    return z


def tone(n: int, k0: int, amp: float) -> np.ndarray:
    """amp * exp(+2 pi i k0 t / n), t = 0 .. n-1, with the phase index reduced
    mod n in integers so that large n keep full accuracy (FP64 complex)."""
    t = (np.int64(k0) * np.arange(n, dtype=np.int64)) % n
    return amp * np.exp(2j * np.pi * t / n)


def tone_2d(nx: int, ny: int, k1: int, k2: int, amp: float) -> np.ndarray:
    """amp * exp(+2 pi i (k1 t1 / nx + k2 t2 / ny)) on an nx x ny grid."""
    return tone(nx, k1, 1.0)[:, None] * tone(ny, k2, amp)[None, :]

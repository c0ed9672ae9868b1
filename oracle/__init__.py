"""FP64 CPU oracle for the tcFFT method (arXiv 2104.11471) -- test infrastructure.

Only the test suite, the package smoke check and the benchmark's CPU-baseline
leg may import this package.  The GPU library never calls it and shares no
code with it.  The arithmetic lives in ``fft_oracle.c`` (plain C, double
precision); this module compiles it with gcc on first use and wraps it with
ctypes.  Every function takes and returns numpy ``complex128`` arrays.

Functions and the passage each one follows:
  dft_brute(x)            Eq. (dft_def), Sec. 2.1: the DFT by its definition.
  dft_bins(x, bins)       Eq. (dft_def) evaluated at selected output bins.
  fft_radix2(x)           Eq. (dft_s2) with N1 = 2, applied recursively.
  fft_mixed(x, radices)   Eq. (dft_mm) merges with the given radices.
  merge(xin)              one merging process, Eq. (dft_mm).
  fft_batch(x)            batched 1D transforms (rows of a 2D array).
  fft_2d(x)               batched 2D transforms, rows then columns (Sec. 3.1).
  twiddle(a, n)           W_n^a = exp(-2 pi i a / n) with integer reduction.
Error metrics (Sec. 5.1, Eq. (prec_def), plus rel-L2 and max-abs):
  rel_l2, max_abs, mean_rel_err.

Parity pins: every function above is checked in tests/test_oracle.py against
closed forms, invariants, brute force and numpy.fft; none is unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fft_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile fft_oracle.c into liboracle.so next to it (gcc, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-D_GNU_SOURCE", "-o", tmp, _SRC,
               "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _bind(lib):
    i64, dp, ip = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
    lib.oracle_dft_brute.argtypes = [i64, dp, dp]
    lib.oracle_dft_bins.argtypes = [i64, dp, i64, dp, dp, ip]
    lib.oracle_fft_radix2.argtypes = [i64, dp, dp]
    lib.oracle_merge.argtypes = [i64, i64, dp, dp]
    lib.oracle_fft_mixed.argtypes = [i64, dp, ip, dp, dp]
    lib.oracle_fft_mixed.restype = ctypes.c_int
    lib.oracle_fft_batch.argtypes = [i64, i64, dp, dp, ip]
    lib.oracle_fft_2d.argtypes = [i64, i64, i64, dp, dp, ip]
    lib.oracle_twiddle.argtypes = [i64, i64, dp]
    for f in (lib.oracle_dft_brute, lib.oracle_dft_bins, lib.oracle_fft_radix2,
              lib.oracle_merge, lib.oracle_fft_batch, lib.oracle_fft_2d, lib.oracle_twiddle):
        f.restype = None
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(_LIB))
    return _lib


def planted_variant(plant: int, out_dir: str):
    """Compile the oracle with a deliberately planted mistake (-DORACLE_PLANT=plant).

    Used only by the mutation tests, which check that the pins in the test
    suite catch each planted mistake.  Returns a module-like object exposing
    the same functions as this package.
    """
    path = os.path.join(out_dir, f"liboracle_plant{plant}.so")
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-std=c99", "-D_GNU_SOURCE",
                    f"-DORACLE_PLANT={int(plant)}", "-o", path, _SRC, "-lm", "-lpthread"],
                   check=True)
    lib = _bind(ctypes.CDLL(path))

    class _Variant:
        pass

    v = _Variant()
    for name in ("twiddle", "dft_brute", "dft_bins", "fft_radix2", "merge", "fft_mixed",
                 "fft_batch", "fft_2d"):
        fn = globals()[name]
        setattr(v, name, (lambda f: (lambda *a, **k: f(*a, _lib_override=lib, **k)))(fn))
    return v


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def _c128(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.complex128))


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _check_pow2(n: int):
    if n < 1 or (n & (n - 1)):
        raise ValueError(f"length {n} is not a power of two")


def twiddle(a: int, n: int, _lib_override=None) -> complex:
    out = np.zeros(2, dtype=np.float64)
    (_lib_override or _load()).oracle_twiddle(int(a), int(n), _ptr(out))
    return complex(out[0], out[1])


def dft_brute(x, _lib_override=None) -> np.ndarray:
    x = _c128(x)
    out = np.empty_like(x)
    (_lib_override or _load()).oracle_dft_brute(x.shape[-1], _ptr(x), _ptr(out))
    return out


def dft_bins(x, bins, nthreads: int | None = None, _lib_override=None) -> np.ndarray:
    x = _c128(x)
    b = np.ascontiguousarray(np.asarray(bins, dtype=np.int64))
    out = np.empty(b.shape[0], dtype=np.complex128)
    (_lib_override or _load()).oracle_dft_bins(x.shape[-1], _ptr(x), b.shape[0], _ptr(b), _ptr(out),
                            nthreads or default_threads())
    return out


def fft_radix2(x, _lib_override=None) -> np.ndarray:
    x = _c128(x)
    _check_pow2(x.shape[-1])
    out = np.empty_like(x)
    (_lib_override or _load()).oracle_fft_radix2(x.shape[-1], _ptr(x), _ptr(out))
    return out


def merge(xin, _lib_override=None) -> np.ndarray:
    """One merging process: xin is the N1 x N2 matrix X_in, returns X_out."""
    xin = _c128(xin)
    n1, n2 = xin.shape
    out = np.empty_like(xin)
    (_lib_override or _load()).oracle_merge(n1, n2, _ptr(xin), _ptr(out))
    return out


def fft_mixed(x, radices, _lib_override=None) -> np.ndarray:
    x = _c128(x)
    r = np.ascontiguousarray(np.asarray(radices, dtype=np.int64))
    out = np.empty_like(x)
    rc = (_lib_override or _load()).oracle_fft_mixed(x.shape[-1], _ptr(r), r.shape[0], _ptr(x), _ptr(out))
    if rc != 0:
        raise ValueError(f"radices {list(radices)} do not multiply to {x.shape[-1]}")
    return out


def fft_batch(x, nthreads: int | None = None, _lib_override=None) -> np.ndarray:
    """x: [batch, n] (or [n]); n-point transform of every row."""
    x = _c128(x)
    n = x.shape[-1]
    _check_pow2(n)
    batch = x.size // n
    out = np.empty_like(x)
    (_lib_override or _load()).oracle_fft_batch(n, batch, _ptr(x), _ptr(out), nthreads or default_threads())
    return out


def fft_2d(x, nthreads: int | None = None, _lib_override=None) -> np.ndarray:
    """x: [batch, nx, ny] (or [nx, ny]), row-major, ny contiguous."""
    x = _c128(x)
    nx, ny = x.shape[-2], x.shape[-1]
    _check_pow2(nx)
    _check_pow2(ny)
    batch = x.size // (nx * ny)
    out = np.empty_like(x)
    (_lib_override or _load()).oracle_fft_2d(nx, ny, batch, _ptr(x), _ptr(out), nthreads or default_threads())
    return out


# ------------------------------------------------------------------ metrics
def rel_l2(got, ref) -> float:
    """||got - ref||_2 / ||ref||_2 over all elements."""
    got = np.asarray(got, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    den = np.linalg.norm(ref.ravel())
    return float(np.linalg.norm((got - ref).ravel()) / (den if den > 0 else 1.0))


def rel_l2_per_row(got, ref) -> np.ndarray:
    got = np.asarray(got, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    n = ref.shape[-1] if ref.ndim == 2 else ref.shape[-1] * ref.shape[-2]
    g = got.reshape(-1, n)
    r = ref.reshape(-1, n)
    den = np.linalg.norm(r, axis=1)
    den[den == 0] = 1.0
    return np.linalg.norm(g - r, axis=1) / den


def max_abs(got, ref) -> float:
    return float(np.max(np.abs(np.asarray(got) - np.asarray(ref)))) if np.size(ref) else 0.0


def mean_rel_err(got, ref, floor: float = 1e-12) -> float:
    """Eq. (prec_def): (1/N) sum_i |X_ref[i] - X[i]| / |X_ref[i]|.

    The printed denominator is garbled; it is read as |X_ref[i]| per element.
    Bins with |X_ref| below floor * max|X_ref| are skipped.
    """
    got = np.asarray(got, dtype=np.complex128).ravel()
    ref = np.asarray(ref, dtype=np.complex128).ravel()
    mag = np.abs(ref)
    keep = mag > floor * (mag.max() if mag.size else 0.0)
    if not np.any(keep):
        return 0.0
    return float(np.mean(np.abs(ref[keep] - got[keep]) / mag[keep]))

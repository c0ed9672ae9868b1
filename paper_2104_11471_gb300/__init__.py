"""Python binding of libtcfft (include/tcfft.h): batched FP16 FFTs on GB300 tensor cores.

The functions below carry the C ABI's names and only marshal arguments:
every step of a transform runs in the CUDA kernels of libtcfft.so.  There is
no fallback -- if the library is missing or no sm_103a GPU is present the
calls raise.  PyTorch is used by callers only for device memory and streams:
``Plan.exec`` accepts CUDA tensors and the current torch stream.

Data layout (see include/tcfft.h): interleaved complex FP16.  A torch
tensor of shape [..., 2] and dtype float16 (re, im), or dtype complex32
("chalf"), holds it; split precision uses a buffer of two such planes.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtcfft.so")

TCFFT_FP16 = 0
TCFFT_FP16_SPLIT = 1
TCFFT_FP32 = 2          # interleaved FP32 complex in and out (split FP16 tensor-core stages)
TCFFT_PLAN_AUTOTUNE = 1
TCFFT_PLAN_GRAPH = 2
TCFFT_PLAN_INVERSE = 4
TCFFT_PLAN_SCALE = 8
TCFFT_PLAN_SHARE_SM = 16  # at most half of each SM's CTA slots (room for other streams)
TCFFT_PLAN_FUSED_2D = 32  # square 2D up to 512^2: rows and columns in one cluster launch
TCFFT_PLAN_PERSISTENT = 64  # ragged plans: one persistent launch over a device work queue

STATUS = {
    0: "TCFFT_OK", 1: "TCFFT_ERR_INVALID_SIZE", 2: "TCFFT_ERR_INVALID_VALUE",
    3: "TCFFT_ERR_ALLOC", 4: "TCFFT_ERR_LAUNCH", 5: "TCFFT_ERR_TIMEOUT",
    6: "TCFFT_ERR_UNSUPPORTED", 7: "TCFFT_ERR_NOT_IMPLEMENTED", 8: "TCFFT_ERR_CUDA",
}

# every function declared in include/tcfft.h: name -> (restype, argtypes)
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_SIG = {
    "tcfft_plan_1d": (ctypes.c_int, [ctypes.POINTER(_P), _I64, _I64]),
    "tcfft_plan_2d": (ctypes.c_int, [ctypes.POINTER(_P), _I64, _I64, _I64]),
    "tcfft_plan_1d_ex": (ctypes.c_int, [ctypes.POINTER(_P), _I64, _I64, ctypes.c_int, ctypes.c_uint]),
    "tcfft_plan_2d_ex": (ctypes.c_int, [ctypes.POINTER(_P), _I64, _I64, _I64, ctypes.c_int, ctypes.c_uint]),
    "tcfft_plan_many": (ctypes.c_int, [ctypes.POINTER(_P), _I64, _P, _P, ctypes.c_int, ctypes.c_uint]),
    "tcfft_exec": (ctypes.c_int, [_P, _P, _P, _P]),
    "tcfft_exec_host": (ctypes.c_int, [_P, _P, _P, _P]),
    "tcfft_exec_batch": (ctypes.c_int, [_P, _P, _P, _I64, _P]),
    "tcfft_destroy": (ctypes.c_int, [_P]),
    "tcfft_plan_last_error": (ctypes.c_int, [_P]),
    "tcfft_io_bytes": (ctypes.c_size_t, [_P]),
    "tcfft_workspace_bytes": (ctypes.c_size_t, [_P]),
    "tcfft_plan_num_launches": (ctypes.c_int, [_P]),
    "tcfft_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "tcfft_plan_describe": (ctypes.c_size_t, [_P, ctypes.c_char_p, ctypes.c_size_t]),
    "tcfft_exec_1d_noalloc": (ctypes.c_int, [_I64, _I64, _P, _P, _P]),
    "tcfft_selftest_wait_timeout": (ctypes.c_int, [ctypes.c_longlong]),
    "tcfft_selftest_queue_timeout": (ctypes.c_int, [ctypes.c_longlong]),
}

_lock = threading.Lock()
_lib = None


class TcfftError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}" if what else STATUS.get(status, str(status)))


def build(force: bool = False) -> str:
    from . import builder
    return builder.build(force=force)


def lib():
    """Load libtcfft.so (built in-tree by build()); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libtcfft.so not built ({LIB_PATH}); run __graft_entry__.build()")
            # torch ships the CUDA runtime the library was linked against
            try:
                import torch  # noqa: F401
            except Exception:
                pass
            h = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIG.items():
                f = getattr(h, name)
                f.restype = res
                f.argtypes = args
            _lib = h
    return _lib


def _check(st: int, what: str):
    if st != 0:
        raise TcfftError(st, what)


# ---------------------------------------------------------------- raw ABI
def tcfft_plan_1d(n: int, batch: int, precision: int = TCFFT_FP16, flags: int = 0) -> int:
    h = _P()
    _check(lib().tcfft_plan_1d_ex(ctypes.byref(h), n, batch, precision, flags), "tcfft_plan_1d")
    return h.value


def tcfft_plan_2d(nx: int, ny: int, batch: int, precision: int = TCFFT_FP16, flags: int = 0) -> int:
    h = _P()
    _check(lib().tcfft_plan_2d_ex(ctypes.byref(h), nx, ny, batch, precision, flags), "tcfft_plan_2d")
    return h.value


def tcfft_plan_many(shapes, precision: int = TCFFT_FP16, flags: int = 0) -> int:
    """shapes: sequence of (n,) or (nx, ny) tuples, packed in that order."""
    cnt = len(shapes)
    a = (ctypes.c_int64 * cnt)(*[s[0] for s in shapes])
    b = (ctypes.c_int64 * cnt)(*[(s[1] if len(s) > 1 else 0) for s in shapes])
    h = _P()
    _check(lib().tcfft_plan_many(ctypes.byref(h), cnt, ctypes.cast(a, _P), ctypes.cast(b, _P), precision, flags),
           "tcfft_plan_many")
    return h.value


def tcfft_exec(plan: int, in_ptr: int, out_ptr: int, stream: int = 0) -> None:
    _check(lib().tcfft_exec(plan, in_ptr, out_ptr, stream), "tcfft_exec")


def tcfft_exec_batch(plan: int, in_ptr: int, out_ptr: int, batch: int, stream: int = 0) -> None:
    _check(lib().tcfft_exec_batch(plan, in_ptr, out_ptr, batch, stream), "tcfft_exec_batch")


def tcfft_exec_host(plan: int, host_in: int, host_out: int, stream: int = 0) -> None:
    _check(lib().tcfft_exec_host(plan, host_in, host_out, stream), "tcfft_exec_host")


def tcfft_exec_1d_noalloc(n: int, batch: int, in_ptr: int, out_ptr: int, stream: int = 0) -> None:
    """Allocation-free 1D transform (see include/tcfft.h): no plan, no device allocation."""
    _check(lib().tcfft_exec_1d_noalloc(n, batch, in_ptr, out_ptr, stream), "tcfft_exec_1d_noalloc")


def tcfft_destroy(plan: int) -> None:
    _check(lib().tcfft_destroy(plan), "tcfft_destroy")


def tcfft_plan_last_error(plan: int) -> int:
    return lib().tcfft_plan_last_error(plan)


def tcfft_io_bytes(plan: int) -> int:
    return lib().tcfft_io_bytes(plan)


def tcfft_workspace_bytes(plan: int) -> int:
    return lib().tcfft_workspace_bytes(plan)


def tcfft_plan_num_launches(plan: int) -> int:
    return lib().tcfft_plan_num_launches(plan)


def tcfft_plan_describe(plan: int) -> list:
    import json
    n = lib().tcfft_plan_describe(plan, None, 0)
    buf = ctypes.create_string_buffer(n)
    lib().tcfft_plan_describe(plan, buf, n)
    return json.loads(buf.value.decode())


def tcfft_status_string(status: int) -> str:
    return lib().tcfft_status_string(status).decode()


# ---------------------------------------------------------------- helpers
def _ptr(t) -> int:
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Plan:
    """Owns a tcfft plan; exec() runs it on CUDA tensors (or raw pointers)."""

    def __init__(self, handle: int, kind: str, shape: tuple, batch: int, precision: int):
        self.handle = handle
        self.kind = kind
        self.shape = shape
        self.batch = batch
        self.precision = precision

    @classmethod
    def plan_1d(cls, n: int, batch: int, precision: int = TCFFT_FP16, flags: int = 0) -> "Plan":
        return cls(tcfft_plan_1d(n, batch, precision, flags), "1d", (n,), batch, precision)

    @classmethod
    def plan_2d(cls, nx: int, ny: int, batch: int, precision: int = TCFFT_FP16, flags: int = 0) -> "Plan":
        return cls(tcfft_plan_2d(nx, ny, batch, precision, flags), "2d", (nx, ny), batch, precision)

    @classmethod
    def plan_many(cls, shapes, precision: int = TCFFT_FP16, flags: int = 0) -> "Plan":
        return cls(tcfft_plan_many(shapes, precision, flags), "many", tuple(shapes), len(shapes), precision)

    @property
    def io_bytes(self) -> int:
        return tcfft_io_bytes(self.handle)

    @property
    def workspace_bytes(self) -> int:
        return tcfft_workspace_bytes(self.handle)

    @property
    def num_launches(self) -> int:
        return tcfft_plan_num_launches(self.handle)

    def describe(self) -> list:
        return tcfft_plan_describe(self.handle)

    def exec(self, inp, out, stream=None) -> None:
        for t in (inp, out):
            if not isinstance(t, int):
                if not t.is_cuda:
                    raise ValueError("tcfft exec needs CUDA tensors")
                if t.numel() * t.element_size() < self.io_bytes:
                    raise ValueError("buffer smaller than the plan's io_bytes")
        tcfft_exec(self.handle, _ptr(inp), _ptr(out), _stream_handle(stream))

    def exec_batch(self, inp, out, batch: int, stream=None) -> None:
        tcfft_exec_batch(self.handle, _ptr(inp), _ptr(out), batch, _stream_handle(stream))

    def exec_host(self, host_in, host_out, stream=None) -> None:
        tcfft_exec_host(self.handle, _ptr(host_in), _ptr(host_out), _stream_handle(stream))

    def last_error(self) -> int:
        return tcfft_plan_last_error(self.handle)

    def destroy(self) -> None:
        if self.handle:
            tcfft_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

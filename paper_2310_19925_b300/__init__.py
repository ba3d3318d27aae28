"""orand-b300: counter-based random number generation on B300 (sm_103a).

Thin Python binding over ``liborand.so`` (the C ABI declared in
``include/orand.h``).  Every computation runs in the library's CUDA kernels;
this module only marshals arguments (raw device pointers from torch tensors,
the current CUDA stream) and turns negative status codes into exceptions.
There is no CPU fallback: if the library is missing, every call raises.

The raw entry points keep the C names (``orand_fill_u32`` ...).  The torch
conveniences (``fill``, ``brownian_walk`` ...) allocate outputs with torch and
call the same entry points.
"""
from __future__ import annotations

import ctypes
import os

from .workloads import (  # noqa: F401  (re-exported enums)
    PHILOX, THREEFRY, SQUARES, TYCHE, U32, F32_UNIFORM, F64_UNIFORM, F32_NORMAL, GEN_NAMES, DTYPE_NAMES,
)

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liborand.so")

ORAND_OK = 0
STATUS_NAMES = {
    0: "ORAND_OK", -1: "ORAND_ERR_INVALID_ARG", -2: "ORAND_ERR_OVERFLOW", -3: "ORAND_ERR_ALIGNMENT",
    -4: "ORAND_ERR_ALLOC", -5: "ORAND_ERR_CUDA", -6: "ORAND_ERR_DEVICE_TIMEOUT", -7: "ORAND_ERR_UNSUPPORTED",
}


class OrandError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib().orand_status_string(status).decode() if _LIB is not None else STATUS_NAMES.get(status, "?")
        if status == -5 and _LIB is not None:
            msg += " (cudaError %d)" % _LIB.orand_last_cuda_error()
        super().__init__("%s: %s" % (where, msg))


_LIB = None

_u64, _u32, _i32, _vp, _sz = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t
_f32, _f64 = ctypes.c_float, ctypes.c_double

# Signatures of the C ABI: name -> (restype, argtypes).
_SIGS = {
    "orand_status_string": (ctypes.c_char_p, [_i32]),
    "orand_version": (_i32, []),
    "orand_last_cuda_error": (_i32, []),
    "orand_fill": (_i32, [_i32, _i32, _u64, _u32, _u64, _u64, _vp, _vp]),
    "orand_fill_u32": (_i32, [_i32, _u64, _u32, _u64, _u64, _vp, _vp]),
    "orand_fill_uniform_f32": (_i32, [_i32, _u64, _u32, _u64, _u64, _vp, _vp]),
    "orand_fill_uniform_f64": (_i32, [_i32, _u64, _u32, _u64, _u64, _vp, _vp]),
    "orand_fill_normal_f32": (_i32, [_i32, _u64, _u32, _u64, _u64, _vp, _vp]),
}


def _lib():
    """Load liborand.so (built in-tree by ``python -m paper_2310_19925_b300.build``)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("liborand.so is not built (%s); run `python -m paper_2310_19925_b300.build`"
                               % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def _check(status: int, where: str):
    if status != ORAND_OK:
        raise OrandError(status, where)


def _stream_handle(stream=None) -> int:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


# ---------------------------------------------------------------- raw C ABI --

def orand_fill(gen, dtype, seed, counter, n_streams, draws_per_stream, out_ptr, stream_handle):
    _check(_lib().orand_fill(gen, dtype, seed & (2**64 - 1), counter & 0xFFFFFFFF, n_streams,
                             draws_per_stream, out_ptr, stream_handle), "orand_fill")


def orand_fill_u32(gen, seed, counter, n_streams, draws_per_stream, out_ptr, stream_handle):
    _check(_lib().orand_fill_u32(gen, seed & (2**64 - 1), counter & 0xFFFFFFFF, n_streams, draws_per_stream,
                                 out_ptr, stream_handle), "orand_fill_u32")


def orand_fill_uniform_f32(gen, seed, counter, n_streams, draws_per_stream, out_ptr, stream_handle):
    _check(_lib().orand_fill_uniform_f32(gen, seed & (2**64 - 1), counter & 0xFFFFFFFF, n_streams,
                                         draws_per_stream, out_ptr, stream_handle), "orand_fill_uniform_f32")


def orand_fill_uniform_f64(gen, seed, counter, n_streams, draws_per_stream, out_ptr, stream_handle):
    _check(_lib().orand_fill_uniform_f64(gen, seed & (2**64 - 1), counter & 0xFFFFFFFF, n_streams,
                                         draws_per_stream, out_ptr, stream_handle), "orand_fill_uniform_f64")


def orand_fill_normal_f32(gen, seed, counter, n_streams, draws_per_stream, out_ptr, stream_handle):
    _check(_lib().orand_fill_normal_f32(gen, seed & (2**64 - 1), counter & 0xFFFFFFFF, n_streams,
                                        draws_per_stream, out_ptr, stream_handle), "orand_fill_normal_f32")


# ----------------------------------------------------------- torch helpers --

def torch_dtype(dtype: int):
    """Storage dtype of a fill's output (u32 words are stored as int32 bit patterns)."""
    import torch

    return {U32: torch.int32, F32_UNIFORM: torch.float32, F64_UNIFORM: torch.float64,
            F32_NORMAL: torch.float32}[dtype]


def fill(gen: int, dtype: int, seed: int, counter: int, n_streams: int, draws_per_stream: int, out=None,
         device="cuda", stream=None):
    """Bulk fill into a (new or given) CUDA tensor of n_streams*draws_per_stream values."""
    import torch

    n = n_streams * draws_per_stream
    if out is None:
        out = torch.empty(n, dtype=torch_dtype(dtype), device=device)
    if out.numel() < n or not out.is_cuda or not out.is_contiguous():
        raise ValueError("out must be a contiguous CUDA tensor with at least %d elements" % n)
    orand_fill(gen, dtype, seed, counter, n_streams, draws_per_stream, _ptr(out) if n else 0,
               _stream_handle(stream))
    return out

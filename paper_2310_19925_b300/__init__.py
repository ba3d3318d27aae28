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
    -8: "ORAND_ERR_SCRATCH_LIMIT",
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
    "orand_fill_streams": (_i32, [_i32, _i32, _u64, _u32, _u64, _u64, _u64, _vp, _vp]),
    "orand_fill_u32": (_i32, [_i32, _u64, _u32, _u64, _u64, _vp, _vp]),
    "orand_fill_uniform_f32": (_i32, [_i32, _u64, _u32, _u64, _u64, _vp, _vp]),
    "orand_fill_uniform_f64": (_i32, [_i32, _u64, _u32, _u64, _u64, _vp, _vp]),
    "orand_fill_normal_f32": (_i32, [_i32, _u64, _u32, _u64, _u64, _vp, _vp]),
    "orand_map_words": (_i32, [_i32, _vp, _u64, _vp, _vp]),
    "orand_engine_draws": (_i32, [_i32, _u64, _u32, _u32, _u64, _u32, _vp, _vp]),
    "orand_host_engine_words": (_i32, [_i32, _u64, _u32, _u32, _u64, _vp]),
    "orand_ctx_create": (_i32, [ctypes.POINTER(_vp)]),
    "orand_ctx_destroy": (_i32, [_vp]),
    "orand_brownian_walk": (_i32, [_vp, _vp, _vp]),
    "orand_walk_normals": (_i32, [_vp, _u64, _vp, _vp]),
    "orand_walk2d_curand_state_bytes": (_sz, []),
    "orand_walk2d_curand_setup": (_i32, [_vp, _vp, _vp, _u64, _vp]),
    "orand_walk2d_curand_run": (_i32, [_vp, _vp, _vp, _vp]),
    "orand_walk2d_curand_fused": (_i32, [_vp, _vp, _u64, _vp]),
    "orand_walk3d_init": (_i32, [_vp, _vp, _vp]),
    "orand_walk3d_fwd": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "orand_walk3d_bwd": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "orand_walk3d_bwd_noalloc": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "orand_walk3d_plain_fwd": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "orand_walk3d_plain_bwd": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "orand_walk3d_stored_fwd": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "orand_walk3d_stored_bwd": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "orand_langevin2d_init": (_i32, [_vp, _vp, _vp]),
    "orand_langevin2d_step": (_i32, [_vp, _vp, _u32, _vp]),
    "orand_langevin2d_fused": (_i32, [_vp, _vp, _u32, _u32, _vp]),
    "orand_langevin2d_run_per_step": (_i32, [_vp, _vp, _u32, _u32, _vp]),
    "orand_langevin2d_curand_run": (_i32, [_vp, _vp, _vp, _u32, _vp]),
    "orand_langevin2d_curand_state_bytes": (_sz, []),
    "orand_langevin2d_curand_setup": (_i32, [_vp, _vp, _vp, _u64, _vp]),
    "orand_langevin2d_curand_step": (_i32, [_vp, _vp, _vp, _vp]),
    "orand_fill_ragged": (_i32, [_vp, _vp, _sz, _vp, _u64, _vp]),
    "orand_fill_micro_streams": (_i32, [_i32, _u64, _u64, _u32, _u32, _u32, _vp, _vp]),
    "orand_stat_tuples": (_i32, [_vp, _u64, _u32, _u32, _u32, _u32, _vp, _vp]),
    "orand_stat_gaps": (_i32, [_vp, _vp, _u64, _u64, _u64, _u32, _vp, _vp, _vp]),
    "orand_stat_birthday": (_i32, [_vp, _u64, _u32, _u32, _u32, _u32, _vp, _vp]),
    "orand_host_fill_u32": (_i32, [_i32, _u64, _u32, _u64, _u64, _vp]),
    "orand_host_microbench": (_i32, [_i32, _vp, _u32, _u64, _vp, _vp]),
    "orand_fill_ragged_serial": (_i32, [_vp, _sz, _vp, _u64, _vp]),
    "orand_ragged_set_config": (_i32, [_vp, _vp]),
    "orand_ragged_get_config": (_i32, [_vp, _vp]),
    "orand_ragged_stats": (_i32, [_vp, _vp]),
}


class RaggedConfig(ctypes.Structure):
    """orand_ragged_config_t."""
    _fields_ = [("block", _u32), ("chunk_values", _u32), ("store_bytes", _u32), ("ctas_per_sm", _u32)]


class RaggedStats(ctypes.Structure):
    """orand_ragged_stats_t."""
    _fields_ = [("graph_launches", _u64), ("graph_builds", _u64), ("tune_runs", _u64), ("tuned_classes", _u64)]


class Walk2DParams(ctypes.Structure):
    """orand_walk2d_t."""
    _fields_ = [("n_particles", _u64), ("p_first", _u64), ("seed", _u64), ("steps", _u32),
                ("dt", _f32), ("D", _f32), ("reserved", _u32)]


class Walk3DParams(ctypes.Structure):
    """orand_walk3d_t."""
    _fields_ = [("n_particles", _u64), ("p_first", _u64), ("p_total", _u64), ("seed", _u64),
                ("steps", _u32), ("ckpt_every", _u32), ("dt", _f32), ("mu", _f32 * 3), ("sigma", _f32),
                ("k", _f32), ("kappa", _f32), ("reserved", _u32)]


class Langevin2DParams(ctypes.Structure):
    """orand_langevin2d_t."""
    _fields_ = [("n_particles", _u64), ("p_first", _u64), ("seed", _u64), ("dt", _f64), ("gamma", _f64),
                ("mass", _f64)]


PARTICLE_BYTES = 40  # orand_particle_t: x, y, vx, vy (double), pid (uint64)

assert ctypes.sizeof(Walk2DParams) == 40 and ctypes.sizeof(Walk3DParams) == 72


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

class Context:
    """An orand_ctx_t: device scratch, ragged tuning table and graph cache."""

    def __init__(self):
        h = _vp()
        _check(_lib().orand_ctx_create(ctypes.byref(h)), "orand_ctx_create")
        self.handle = h.value

    def close(self):
        if self.handle:
            _check(_lib().orand_ctx_destroy(self.handle), "orand_ctx_destroy")
            self.handle = None


_CONTEXTS = {}


def default_context(device=None) -> Context:
    """One library context per device, created on first use and kept for the process."""
    import torch

    dev = torch.cuda.current_device() if device is None else int(device)
    if dev not in _CONTEXTS:
        with torch.cuda.device(dev):
            _CONTEXTS[dev] = Context()
    return _CONTEXTS[dev]


def orand_fill(gen, dtype, seed, counter, n_streams, draws_per_stream, out_ptr, stream_handle):
    _check(_lib().orand_fill(gen, dtype, seed & (2**64 - 1), counter & 0xFFFFFFFF, n_streams,
                             draws_per_stream, out_ptr, stream_handle), "orand_fill")


def orand_fill_streams(gen, dtype, seed, counter, first_stream, n_streams, draws_per_stream, out_ptr,
                       stream_handle):
    _check(_lib().orand_fill_streams(gen, dtype, seed & (2**64 - 1), counter & 0xFFFFFFFF, first_stream,
                                     n_streams, draws_per_stream, out_ptr, stream_handle), "orand_fill_streams")


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


def orand_map_words(dtype, words_ptr, n_values, out_ptr, stream_handle):
    _check(_lib().orand_map_words(dtype, words_ptr, n_values, out_ptr, stream_handle), "orand_map_words")


# ----------------------------------------------------------- torch helpers --

def torch_dtype(dtype: int):
    """Storage dtype of a fill's output (u32 words are stored as int32 bit patterns)."""
    import torch

    return {U32: torch.int32, F32_UNIFORM: torch.float32, F64_UNIFORM: torch.float64,
            F32_NORMAL: torch.float32}[dtype]


def map_words(dtype: int, words, n_values=None, stream=None):
    """Apply a dtype's word->value map to a CUDA int32 tensor of words."""
    import torch

    if n_values is None:
        n_values = words.numel() // 2 if dtype == F64_UNIFORM else words.numel()
    out = torch.empty(n_values, dtype=torch_dtype(dtype), device=words.device)
    orand_map_words(dtype, _ptr(words), n_values, _ptr(out) if n_values else 0, _stream_handle(stream))
    return out


def fill(gen: int, dtype: int, seed: int, counter: int, n_streams: int, draws_per_stream: int, out=None,
         device="cuda", stream=None, first_stream: int = 0):
    """Bulk fill into a (new or given) CUDA tensor of n_streams*draws_per_stream
    values: streams first_stream .. first_stream + n_streams - 1 of the fill
    keyed by seed."""
    import torch

    n = n_streams * draws_per_stream
    if out is None:
        out = torch.empty(n, dtype=torch_dtype(dtype), device=device)
    if out.numel() < n or not out.is_cuda or not out.is_contiguous():
        raise ValueError("out must be a contiguous CUDA tensor with at least %d elements" % n)
    if first_stream:
        orand_fill_streams(gen, dtype, seed, counter, first_stream, n_streams, draws_per_stream,
                           _ptr(out) if n else 0, _stream_handle(stream))
    else:
        orand_fill(gen, dtype, seed, counter, n_streams, draws_per_stream, _ptr(out) if n else 0,
                   _stream_handle(stream))
    return out


# ------------------------------------------------- per-thread engines --

# One round of orand_engine_draws (48 bytes): the draws in the order
# w, d1, n, u, d2, u2; stored d2, d1, n, u2, w, u.
ENGINE_RECORD_FIELDS = [("d2", "<f8", (2,)), ("d1", "<f8"), ("n", "<f4", (2,)), ("u2", "<f4", (2,)),
                        ("w", "<u4"), ("u", "<f4")]
ENGINE_RECORD_BYTES = 48


def orand_engine_draws(gen, seed, counter, first_word, n_threads, n_rounds, out_ptr, stream_handle):
    _check(_lib().orand_engine_draws(gen, seed & (2**64 - 1), counter & 0xFFFFFFFF, first_word & 0xFFFFFFFF,
                                     n_threads, n_rounds, out_ptr, stream_handle), "orand_engine_draws")


def engine_draws(gen, seed, counter, n_threads, n_rounds, first_word=0, stream=None):
    """Per-thread draws through the device header's engine classes: a CUDA
    uint8 tensor of n_threads * n_rounds 48-byte records (ENGINE_RECORD_FIELDS)."""
    import torch

    out = torch.empty(max(n_threads * n_rounds * ENGINE_RECORD_BYTES, 16), dtype=torch.uint8, device="cuda")
    orand_engine_draws(gen, seed, counter, first_word, n_threads, n_rounds, _ptr(out), _stream_handle(stream))
    return out


def host_engine_words(gen, seed, counter, n, first_word=0):
    """n words of one stream drawn on the host through the engine classes,
    from word first_word (numpy uint32)."""
    import numpy as np

    out = np.empty(n, dtype=np.uint32)
    _check(_lib().orand_host_engine_words(gen, seed & (2**64 - 1), counter & 0xFFFFFFFF, first_word & 0xFFFFFFFF,
                                          n, out.ctypes.data if n else None), "orand_host_engine_words")
    return out


# ------------------------------------------- parallel-stream statistics --

GAP_NO_HIT = 2**64 - 1


def orand_fill_micro_streams(gen, seed, n_streams, draws, counter_first, n_counters, out_ptr, stream_handle):
    _check(_lib().orand_fill_micro_streams(gen, seed & (2**64 - 1), n_streams, draws, counter_first & 0xFFFFFFFF,
                                           n_counters, out_ptr, stream_handle), "orand_fill_micro_streams")


def orand_stat_tuples(words_ptr, n_words, t, bits, shift, stride, counts_ptr, stream_handle):
    _check(_lib().orand_stat_tuples(words_ptr, n_words, t, bits, shift, stride, counts_ptr, stream_handle),
           "orand_stat_tuples")


def orand_stat_gaps(ctx, words_ptr, n_words, lo, hi, t_max, counts_ptr, carry_ptr, stream_handle):
    _check(_lib().orand_stat_gaps(ctx, words_ptr, n_words, lo, hi, t_max, counts_ptr, carry_ptr, stream_handle),
           "orand_stat_gaps")


def orand_stat_birthday(words_ptr, n_words, log2_n, bits, shift, r_max, counts_ptr, stream_handle):
    _check(_lib().orand_stat_birthday(words_ptr, n_words, log2_n, bits, shift, r_max, counts_ptr, stream_handle),
           "orand_stat_birthday")


def fill_micro_streams(gen, seed, n_streams, draws, counter_first, n_counters, out=None, stream=None):
    """The concatenated micro-stream as a CUDA int32 tensor (u32 bits) of
    n_counters * n_streams * draws words."""
    import torch

    n = n_counters * n_streams * draws
    if out is None:
        out = torch.empty(n, dtype=torch.int32, device="cuda")
    if out.numel() < n or not out.is_cuda or not out.is_contiguous():
        raise ValueError("out must be a contiguous CUDA tensor with at least %d elements" % n)
    orand_fill_micro_streams(gen, seed, n_streams, draws, counter_first, n_counters, _ptr(out) if n else 0,
                             _stream_handle(stream))
    return out


def _counts(n, counts):
    import torch

    if counts is None:
        counts = torch.zeros(n, dtype=torch.int64, device="cuda")
    if counts.numel() != n or counts.dtype != torch.int64 or not counts.is_cuda:
        raise ValueError("counts must be a CUDA int64 tensor of %d elements" % n)
    return counts


def _words(words):
    if not words.is_cuda or not words.is_contiguous() or words.element_size() != 4:
        raise ValueError("words must be a contiguous CUDA tensor of 32-bit elements")
    return words


def stat_tuples(words, t, bits, shift, stride, counts=None, stream=None):
    """Accumulate tuple counts (2^(t*bits) int64) of a CUDA u32/int32 tensor."""
    w = _words(words)
    c = _counts(1 << (t * bits), counts)
    orand_stat_tuples(_ptr(w) if w.numel() else 0, w.numel(), t, bits, shift, stride, _ptr(c), _stream_handle(stream))
    return c


def stat_gaps(words, lo, hi, t_max, counts=None, carry=None, stream=None):
    """Accumulate gap counts (t_max + 1 int64); `carry` is a 1-element CUDA
    int64 tensor holding the open run (GAP_NO_HIT bits before the first hit).
    Returns (counts, carry)."""
    import torch

    w = _words(words)
    c = _counts(t_max + 1, counts)
    if carry is None:
        carry = torch.full((1,), -1, dtype=torch.int64, device="cuda")   # all ones = GAP_NO_HIT
    orand_stat_gaps(default_context().handle, _ptr(w) if w.numel() else 0, w.numel(), lo, hi, t_max, _ptr(c),
                    _ptr(carry), _stream_handle(stream))
    return c, carry


def stat_birthday(words, log2_n, bits, shift, r_max, counts=None, stream=None):
    """Accumulate birthday-spacing counts (r_max + 1 int64) over whole samples of 2^log2_n words."""
    w = _words(words)
    c = _counts(r_max + 1, counts)
    orand_stat_birthday(_ptr(w) if w.numel() else 0, w.numel(), log2_n, bits, shift, r_max, _ptr(c),
                        _stream_handle(stream))
    return c


# ------------------------------------------------------------------- host --

HOST_MT19937 = 100


def host_fill_u32(gen, seed, counter, n_streams, draws_per_stream):
    """The u32 fill computed on the host (numpy uint32 array); same bits as
    orand_fill_u32 on the GPU."""
    import numpy as np

    out = np.empty(n_streams * draws_per_stream, dtype=np.uint32)
    _check(_lib().orand_host_fill_u32(gen, seed & (2**64 - 1), counter & 0xFFFFFFFF, n_streams, draws_per_stream,
                                      out.ctypes.data if out.size else None), "orand_host_fill_u32")
    return out


def host_microbench(gen, lengths, words_per_length=1 << 22):
    """ns per stream for each stream length (the paper's host micro-benchmark)."""
    import numpy as np

    L = np.ascontiguousarray(lengths, dtype=np.uint64)
    ns = np.zeros(L.size, dtype=np.float64)
    sink = np.zeros(1, dtype=np.uint32)
    _check(_lib().orand_host_microbench(gen, L.ctypes.data, L.size, words_per_length, ns.ctypes.data,
                                        sink.ctypes.data), "orand_host_microbench")
    return ns


# ------------------------------------------------------------------ walks --

def walk2d_params(n_particles, steps, dt=1e-3, D=1.0, seed=0, p_first=0) -> Walk2DParams:
    return Walk2DParams(n_particles, p_first, seed & (2**64 - 1), steps, dt, D, 0)


def orand_brownian_walk(params: Walk2DParams, pos_out_ptr, stream_handle):
    _check(_lib().orand_brownian_walk(ctypes.byref(params), pos_out_ptr, stream_handle), "orand_brownian_walk")


def orand_walk2d_curand_state_bytes():
    return int(_lib().orand_walk2d_curand_state_bytes())


def orand_walk2d_curand_setup(params, states_ptr, pos_ptr, curand_seed, stream_handle):
    _check(_lib().orand_walk2d_curand_setup(ctypes.byref(params), states_ptr, pos_ptr, curand_seed & (2**64 - 1),
                                            stream_handle), "orand_walk2d_curand_setup")


def orand_walk2d_curand_run(params, states_ptr, pos_ptr, stream_handle):
    _check(_lib().orand_walk2d_curand_run(ctypes.byref(params), states_ptr, pos_ptr, stream_handle),
           "orand_walk2d_curand_run")


def orand_walk2d_curand_fused(params, pos_ptr, curand_seed, stream_handle):
    _check(_lib().orand_walk2d_curand_fused(ctypes.byref(params), pos_ptr, curand_seed & (2**64 - 1),
                                            stream_handle), "orand_walk2d_curand_fused")


def walk_normals(words, stream=None):
    """The walks' Box-Muller map on a CUDA tensor of 2n u32 words (int32 bits): 2n floats."""
    import torch

    w = words.contiguous()
    out = torch.empty(w.numel(), dtype=torch.float32, device="cuda")
    _check(_lib().orand_walk_normals(_ptr(w) if w.numel() else 0, w.numel() // 2, _ptr(out) if w.numel() else 0,
                                     _stream_handle(stream)), "orand_walk_normals")
    return out


def brownian_walk(n_particles, steps, dt=1e-3, D=1.0, seed=0, p_first=0, out=None, stream=None):
    """Fused 2D walk; returns an (n_particles, 2) float32 CUDA tensor of final positions."""
    import torch

    if out is None:
        out = torch.empty((n_particles, 2), dtype=torch.float32, device="cuda")
    orand_brownian_walk(walk2d_params(n_particles, steps, dt, D, seed, p_first), _ptr(out) if n_particles else 0,
                        _stream_handle(stream))
    return out


def walk3d_params(n_particles, steps, dt=1e-3, mu=(0.1, -0.2, 0.05), sigma=0.5, k=2.0, seed=0,
                  ckpt_every=64, p_first=0, p_total=0, kappa=0.0) -> Walk3DParams:
    return Walk3DParams(n_particles, p_first, p_total, seed & (2**64 - 1), steps, ckpt_every, dt,
                        (_f32 * 3)(*[float(m) for m in mu]), float(sigma), float(k), float(kappa), 0)


def n_checkpoints(steps, ckpt_every):
    return 0 if not ckpt_every else (steps + ckpt_every - 1) // ckpt_every


def orand_walk3d_init(params, x0_ptr, stream_handle):
    _check(_lib().orand_walk3d_init(ctypes.byref(params), x0_ptr, stream_handle), "orand_walk3d_init")


def orand_walk3d_fwd(ctx, params, x0_ptr, xT_ptr, ckpt_ptr, loss_ptr, stream_handle):
    _check(_lib().orand_walk3d_fwd(ctx, ctypes.byref(params), x0_ptr, xT_ptr, ckpt_ptr, loss_ptr,
                                   stream_handle), "orand_walk3d_fwd")


def orand_walk3d_bwd(ctx, params, xT_ptr, ckpt_ptr, grad_loss_ptr, dmu_ptr, dsigma_ptr, dkappa_ptr, dx0_ptr,
                     stream_handle):
    _check(_lib().orand_walk3d_bwd(ctx, ctypes.byref(params), xT_ptr, ckpt_ptr, grad_loss_ptr, dmu_ptr, dsigma_ptr,
                                   dkappa_ptr, dx0_ptr, stream_handle), "orand_walk3d_bwd")


def orand_walk3d_bwd_noalloc(params, xT_ptr, ckpt_ptr, grad_loss_ptr, dmu_ptr, dsigma_ptr, dkappa_ptr, dx0_ptr,
                             stream_handle):
    """The adjoint without a context or any allocation (fixed 2^22-particle scratch)."""
    _check(_lib().orand_walk3d_bwd_noalloc(ctypes.byref(params), xT_ptr, ckpt_ptr, grad_loss_ptr, dmu_ptr,
                                           dsigma_ptr, dkappa_ptr, dx0_ptr, stream_handle),
           "orand_walk3d_bwd_noalloc")


def orand_walk3d_plain_fwd(ctx, params, x0_ptr, x_ptr, z_ptr, loss_ptr, stream_handle):
    _check(_lib().orand_walk3d_plain_fwd(ctx, ctypes.byref(params), x0_ptr, x_ptr, z_ptr, loss_ptr,
                                         stream_handle), "orand_walk3d_plain_fwd")


def orand_walk3d_stored_fwd(ctx, params, x0_ptr, xT_ptr, z_store_ptr, loss_ptr, stream_handle):
    _check(_lib().orand_walk3d_stored_fwd(ctx, ctypes.byref(params), x0_ptr, xT_ptr, z_store_ptr, loss_ptr,
                                          stream_handle), "orand_walk3d_stored_fwd")


def orand_walk3d_stored_bwd(ctx, params, xT_ptr, z_store_ptr, grad_loss_ptr, dmu_ptr, dsigma_ptr, dx0_ptr,
                            stream_handle):
    _check(_lib().orand_walk3d_stored_bwd(ctx, ctypes.byref(params), xT_ptr, z_store_ptr, grad_loss_ptr, dmu_ptr,
                                          dsigma_ptr, dx0_ptr, stream_handle), "orand_walk3d_stored_bwd")


def orand_walk3d_plain_bwd(ctx, params, xT_ptr, z_ptr, grad_loss_ptr, dmu_ptr, dsigma_ptr, dx0_ptr,
                           stream_handle):
    _check(_lib().orand_walk3d_plain_bwd(ctx, ctypes.byref(params), xT_ptr, z_ptr, grad_loss_ptr, dmu_ptr,
                                         dsigma_ptr, dx0_ptr, stream_handle), "orand_walk3d_plain_bwd")


def walk3d_init(params: Walk3DParams, stream=None):
    """x0 = 2u - 1 from counter 0 for every particle: (n, 3) float32."""
    import torch

    x0 = torch.empty((params.n_particles, 3), dtype=torch.float32, device="cuda")
    orand_walk3d_init(params, _ptr(x0), _stream_handle(stream))
    return x0


def walk3d_forward(params: Walk3DParams, x0=None, want_ckpt=True, stream=None):
    """Fused forward: returns (xT (n,3) f32, ckpt (C,n,3) f32 or None, loss 0-dim f64)."""
    import torch

    n = params.n_particles
    xT = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    C = n_checkpoints(params.steps, params.ckpt_every) if want_ckpt else 0
    ckpt = torch.empty((C, n, 3), dtype=torch.float32, device="cuda") if C else None
    loss = torch.empty((), dtype=torch.float64, device="cuda")
    if x0 is not None:
        x0 = x0.detach().contiguous()
    orand_walk3d_fwd(default_context().handle, params, _ptr(x0), _ptr(xT), _ptr(ckpt), _ptr(loss),
                     _stream_handle(stream))
    return xT, ckpt, loss


def walk3d_backward(params: Walk3DParams, xT, grad_loss=None, ckpt=None, stream=None):
    """Noise-regenerating adjoint: returns (dmu (3,) f64, dsigma 0-dim f64, dx0 (n,3) f32).
    With kappa != 0 the forward's checkpoints are required."""
    dmu, dsig, _, dx0 = _walk3d_backward(params, xT, grad_loss, ckpt, False, stream)
    return dmu, dsig, dx0


def walk3d_backward_full(params: Walk3DParams, xT, ckpt, grad_loss=None, stream=None):
    """Adjoint including dL/dkappa: returns (dmu, dsigma, dkappa, dx0); needs the checkpoints."""
    return _walk3d_backward(params, xT, grad_loss, ckpt, True, stream)


def _walk3d_backward(params, xT, grad_loss, ckpt, want_dkappa, stream):
    import torch

    dmu = torch.empty(3, dtype=torch.float64, device="cuda")
    dsig = torch.empty((), dtype=torch.float64, device="cuda")
    dkap = torch.empty((), dtype=torch.float64, device="cuda") if want_dkappa else None
    dx0 = torch.empty_like(xT)
    g = None if grad_loss is None else grad_loss.detach().to(device="cuda", dtype=torch.float64).contiguous()
    ck = None if ckpt is None else ckpt.contiguous()
    orand_walk3d_bwd(default_context().handle, params, _ptr(xT.contiguous()), _ptr(ck), _ptr(g), _ptr(dmu),
                     _ptr(dsig), _ptr(dkap), _ptr(dx0), _stream_handle(stream))
    return dmu, dsig, dkap, dx0


def _autograd_function():
    import torch

    class BrownianWalk3D(torch.autograd.Function):
        """loss = BrownianWalk3D.apply(mu, sigma, x0, steps, dt, k, seed, ckpt_every, kappa)

        Forward runs the fused walk with drift mu - kappa x.  It writes
        checkpoints every `ckpt_every` steps; they are saved for backward on
        this call's autograd context only, so they are freed with the graph
        once backward has run (call walk3d_forward directly to keep them).
        Backward runs the adjoint kernel, which regenerates every noise draw
        from its (particle, step) key instead of storing it; for kappa it
        recomputes positions backwards from the checkpoints.

        mu: (3,) tensor; sigma and kappa: 0-dim tensors (each may require
        grad; kappa may be None for 0); x0: (n, 3) CUDA float32.  mu, sigma
        and kappa enter the kernels by value, as kernel parameters: keep
        them on the CPU (their gradients come back on the CPU too), since
        reading a CUDA tensor's value waits for the device.
        """

        @staticmethod
        def forward(ctx, mu, sigma, x0, steps, dt=1e-3, k=2.0, seed=0, ckpt_every=64, kappa=None):
            mu_v = [float(v) for v in mu.detach().reshape(-1).tolist()]
            kap = 0.0 if kappa is None else float(kappa.detach())
            p = walk3d_params(x0.shape[0], int(steps), float(dt), mu_v, float(sigma.detach()), float(k),
                              int(seed), int(ckpt_every), kappa=kap)
            xT, ckpt, loss = walk3d_forward(p, x0=x0, want_ckpt=bool(ckpt_every))
            ctx.params = p
            ctx.want_dkappa = kappa is not None and kappa.requires_grad
            ctx.meta = [(t.dtype, t.device) if t is not None else None for t in (mu, sigma, kappa)]
            if ckpt is None:
                ctx.save_for_backward(xT)
            else:
                ctx.save_for_backward(xT, ckpt)
            return loss

        @staticmethod
        def backward(ctx, grad_loss):
            saved = ctx.saved_tensors
            xT, ckpt = saved[0], (saved[1] if len(saved) > 1 else None)
            dmu, dsig, dkap, dx0 = _walk3d_backward(ctx.params, xT, grad_loss, ckpt, ctx.want_dkappa, None)
            (mdt, mdev), (sdt, sdev) = ctx.meta[0], ctx.meta[1]
            gk = None
            if ctx.want_dkappa:
                gk = dkap.to(dtype=ctx.meta[2][0], device=ctx.meta[2][1])
            return (dmu.to(dtype=mdt, device=mdev), dsig.to(dtype=sdt, device=sdev), dx0,
                    None, None, None, None, None, gk)

    return BrownianWalk3D


_BW3D = None


def BrownianWalk3D():
    """The torch.autograd.Function class for the differentiable 3D walk."""
    global _BW3D
    if _BW3D is None:
        _BW3D = _autograd_function()
    return _BW3D


# ----------------------------------------------------------------- ragged --

def orand_fill_ragged(ctx, reqs_ptr, n, out_base_ptr, out_bytes, stream_handle):
    _check(_lib().orand_fill_ragged(ctx, reqs_ptr, n, out_base_ptr, out_bytes, stream_handle), "orand_fill_ragged")


def orand_fill_ragged_serial(reqs_ptr, n, out_base_ptr, out_bytes, stream_handle):
    _check(_lib().orand_fill_ragged_serial(reqs_ptr, n, out_base_ptr, out_bytes, stream_handle),
           "orand_fill_ragged_serial")


def orand_ragged_set_config(ctx, cfg):
    _check(_lib().orand_ragged_set_config(ctx, None if cfg is None else ctypes.byref(cfg)), "orand_ragged_set_config")


def orand_ragged_get_config(ctx) -> RaggedConfig:
    c = RaggedConfig()
    _check(_lib().orand_ragged_get_config(ctx, ctypes.byref(c)), "orand_ragged_get_config")
    return c


def orand_ragged_stats(ctx) -> RaggedStats:
    st = RaggedStats()
    _check(_lib().orand_ragged_stats(ctx, ctypes.byref(st)), "orand_ragged_stats")
    return st


def fill_ragged(requests, out=None, out_bytes=None, serial=False, ctx=None, stream=None):
    """Serve a ragged batch.  `requests` is a numpy array of
    workloads.REQUEST_DTYPE records (host memory); `out` a CUDA byte buffer
    (allocated when None, sized from the records).  serial=True uses the
    one-launch-per-request baseline.  Returns `out`."""
    import numpy as np
    import torch

    from .workloads import REQUEST_DTYPE, ELEM_BYTES

    reqs = np.ascontiguousarray(requests, dtype=REQUEST_DTYPE)
    if out is None:
        if out_bytes is None:
            ends = [int(r["out_offset_bytes"]) + int(r["length"]) * ELEM_BYTES[int(r["dtype"])] for r in reqs] \
                if len(reqs) < 4096 else (reqs["out_offset_bytes"] + reqs["length"] *
                                          np.where(reqs["dtype"] == 2, 8, 4).astype(np.uint64)).tolist()
            out_bytes = int(max(ends)) if len(reqs) else 0
        out = torch.zeros(max(out_bytes, 1), dtype=torch.uint8, device="cuda")
    nbytes = out.numel() * out.element_size() if out_bytes is None else out_bytes
    sh = _stream_handle(stream)
    if serial:
        orand_fill_ragged_serial(reqs.ctypes.data, len(reqs), _ptr(out), nbytes, sh)
    else:
        c = (ctx or default_context()).handle
        orand_fill_ragged(c, reqs.ctypes.data, len(reqs), _ptr(out), nbytes, sh)
    return out


# -------------------------------------------- paper macro-benchmark (Fig. 1) --

def langevin2d_params(n_particles, dt=1e-3, gamma=1.0, mass=1.0, seed=0, p_first=0) -> Langevin2DParams:
    return Langevin2DParams(n_particles, p_first, seed & (2**64 - 1), dt, gamma, mass)


def orand_langevin2d_init(params, particles_ptr, stream_handle):
    _check(_lib().orand_langevin2d_init(ctypes.byref(params), particles_ptr, stream_handle), "orand_langevin2d_init")


def orand_langevin2d_step(params, particles_ptr, counter, stream_handle):
    _check(_lib().orand_langevin2d_step(ctypes.byref(params), particles_ptr, counter, stream_handle),
           "orand_langevin2d_step")


def orand_langevin2d_fused(params, particles_ptr, first_counter, steps, stream_handle):
    _check(_lib().orand_langevin2d_fused(ctypes.byref(params), particles_ptr, first_counter, steps, stream_handle),
           "orand_langevin2d_fused")


def orand_langevin2d_run_per_step(params, particles_ptr, first_counter, steps, stream_handle):
    _check(_lib().orand_langevin2d_run_per_step(ctypes.byref(params), particles_ptr, first_counter, steps,
                                                stream_handle), "orand_langevin2d_run_per_step")


def orand_langevin2d_curand_run(params, particles_ptr, states_ptr, steps, stream_handle):
    _check(_lib().orand_langevin2d_curand_run(ctypes.byref(params), particles_ptr, states_ptr, steps, stream_handle),
           "orand_langevin2d_curand_run")


def orand_langevin2d_curand_state_bytes() -> int:
    return int(_lib().orand_langevin2d_curand_state_bytes())


def orand_langevin2d_curand_setup(params, particles_ptr, states_ptr, curand_seed, stream_handle):
    _check(_lib().orand_langevin2d_curand_setup(ctypes.byref(params), particles_ptr, states_ptr, curand_seed,
                                                stream_handle), "orand_langevin2d_curand_setup")


def orand_langevin2d_curand_step(params, particles_ptr, states_ptr, stream_handle):
    _check(_lib().orand_langevin2d_curand_step(ctypes.byref(params), particles_ptr, states_ptr, stream_handle),
           "orand_langevin2d_curand_step")


def particles_tensor(n):
    """Device storage for n orand_particle_t (5 x 8 bytes each)."""
    import torch

    return torch.empty((n, 5), dtype=torch.float64, device="cuda")


def particle_state(particles):
    """(x, y, vx, vy) columns of a particle tensor, as a float64 tensor view."""
    return particles[:, :4]

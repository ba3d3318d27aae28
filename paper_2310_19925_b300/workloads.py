"""Seeded synthetic workloads shared by the tests, the smoke check and the benchmark.

This module holds only workload shapes and seeded input generators: no
generator rounds, maps or walk arithmetic.  Its random draws use numpy's
PCG64 (``numpy.random.default_rng``), never one of the library's own
generators, so neither side of a parity check produces the other's inputs.

Workloads (all synthetic; the paper has no dataset):
  * FILL_SMALL   -- Philox4x32-10 bulk fill, global seed 42, 2^16 streams x 64
                    draws, counter 0 (u32 and FP32 uniform).
  * FILL_LARGE   -- all four generators x {u32, FP32 uniform, FP64 uniform,
                    FP32 normal}, 2^24 streams x 16 draws (2^28 values),
                    key64 = stream id ^ 0x5EED, counter 0.
  * WALK2D       -- 2^24 particles, 10,000 steps, dt = 1e-3, D = 1 (the
                    paper's Brownian macro-benchmark of §5 in its
                    pure-diffusion FP32 form).
  * RAGGED       -- 100,000 requests of mixed generator and dtype, lengths
                    log-uniform in [1, 2^20].
  * WALK3D       -- 2^22 particles, 4096 steps, dt = 1e-3,
                    mu = (0.1, -0.2, 0.05), sigma = 0.5, k = 2, checkpoint
                    every 64 steps.
  * WALK3D_OU    -- the same walk with Ornstein-Uhlenbeck drift
                    mu - kappa x, kappa = 1 (the checkpoints carry the
                    adjoint's reverse-time recompute).
"""
from __future__ import annotations

import numpy as np

PHILOX, THREEFRY, SQUARES, TYCHE = 0, 1, 2, 3
U32, F32_UNIFORM, F64_UNIFORM, F32_NORMAL = 0, 1, 2, 3
GEN_NAMES = {PHILOX: "philox4x32_10", THREEFRY: "threefry4x32_20", SQUARES: "squares32", TYCHE: "tyche"}
DTYPE_NAMES = {U32: "u32", F32_UNIFORM: "f32_uniform", F64_UNIFORM: "f64_uniform", F32_NORMAL: "f32_normal"}
ELEM_BYTES = {U32: 4, F32_UNIFORM: 4, F64_UNIFORM: 8, F32_NORMAL: 4}

FILL_SMALL = dict(seed=42, counter=0, n_streams=1 << 16, dps=64)
FILL_LARGE = dict(seed=0x5EED, counter=0, n_streams=1 << 24, dps=16)
WALK2D = dict(n_particles=1 << 24, steps=10_000, dt=1e-3, D=1.0, seed=0)
WALK3D = dict(n_particles=1 << 22, steps=4096, dt=1e-3, mu=(0.1, -0.2, 0.05), sigma=0.5, k=2.0,
              ckpt_every=64, seed=0)
WALK3D_OU = dict(WALK3D, kappa=1.0)
RAGGED = dict(n_requests=100_000, max_log2_len=20, list_seed=20231030)

# Layout of one ragged request record (matches the C struct orand_request_t).
REQUEST_DTYPE = np.dtype([
    ("gen", "<u4"), ("dtype", "<u4"), ("seed", "<u8"), ("counter", "<u4"), ("reserved", "<u4"),
    ("length", "<u8"), ("out_offset_bytes", "<u8"),
])
assert REQUEST_DTYPE.itemsize == 40


def ragged_requests(n_requests: int = RAGGED["n_requests"], max_log2_len: int = RAGGED["max_log2_len"],
                    list_seed: int = RAGGED["list_seed"], dtypes=(U32, F32_UNIFORM, F32_NORMAL),
                    gens=(PHILOX, THREEFRY, SQUARES, TYCHE), align: int = 16):
    """Seeded ragged request list.

    Request i: generator and dtype uniform over ``gens``/``dtypes``; seed = i;
    counter uniform in [0, 2^32); length = floor(2^(max_log2_len * u)) with u
    uniform in [0, 1) (log-uniform in [1, 2^max_log2_len]); outputs packed in
    request order, each start rounded up to ``align`` bytes.  Returns
    (records, total_bytes)."""
    rng = np.random.default_rng(list_seed)
    recs = np.zeros(n_requests, REQUEST_DTYPE)
    recs["gen"] = np.asarray(gens, np.uint32)[rng.integers(0, len(gens), n_requests)]
    recs["dtype"] = np.asarray(dtypes, np.uint32)[rng.integers(0, len(dtypes), n_requests)]
    recs["seed"] = np.arange(n_requests, dtype=np.uint64)
    recs["counter"] = rng.integers(0, 1 << 32, n_requests, dtype=np.uint64).astype(np.uint32)
    u = rng.random(n_requests)
    length = np.floor(np.exp2(max_log2_len * u)).astype(np.uint64)
    recs["length"] = np.clip(length, 1, 1 << max_log2_len)
    elem = np.array([ELEM_BYTES[int(d)] for d in range(4)], np.uint64)[recs["dtype"]]
    nbytes = recs["length"] * elem
    padded = (nbytes + np.uint64(align - 1)) // np.uint64(align) * np.uint64(align)
    offs = np.zeros(n_requests, np.uint64)
    if n_requests > 1:
        offs[1:] = np.cumsum(padded[:-1], dtype=np.uint64)
    recs["out_offset_bytes"] = offs
    total = int(offs[-1] + padded[-1]) if n_requests else 0
    return recs, total


def walk3d_params(**over):
    p = dict(WALK3D)
    p.update(over)
    return p

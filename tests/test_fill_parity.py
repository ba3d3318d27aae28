"""GPU parity of the bulk fills against the CPU oracle.

Bar: u32 words, FP32 and FP64 uniforms bit-exact; FP32 normals within 4 ulp
(ordered-integer distance) of the FP64 oracle value rounded to FP32.  Small
shapes span several groups, ragged tails and both store paths; the full
2^24 x 16 workload runs in the benchmark's launch configuration and is
checked on every value, plus whole-array properties.
"""
import math

import numpy as np
import pytest

from helpers import to_numpy, ulp_distance_f32

import paper_2310_19925_b300 as orand
from paper_2310_19925_b300 import workloads as W

pytestmark = pytest.mark.gpu

GENS = [W.PHILOX, W.THREEFRY, W.SQUARES, W.TYCHE]
DTYPES = [W.U32, W.F32_UNIFORM, W.F64_UNIFORM, W.F32_NORMAL]
NORMAL_ULP = 4


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def compare(dtype, gpu, ref):
    if dtype == W.F32_NORMAL:
        d = ulp_distance_f32(gpu, ref)
        assert d.max(initial=0) <= NORMAL_ULP, "max ulp %d" % d.max()
    elif dtype == W.F32_UNIFORM:
        assert np.array_equal(gpu.astype(np.float64), ref)
    else:
        assert np.array_equal(gpu, ref)


def gpu_fill(torch, gen, dtype, seed, counter, n_streams, dps, offset_elems=0):
    n = n_streams * dps
    buf = torch.full((n + offset_elems + 4,), -7, dtype=orand.torch_dtype(dtype), device="cuda")
    out = buf[offset_elems:offset_elems + n]
    orand.fill(gen, dtype, seed, counter, n_streams, dps, out=out)
    torch.cuda.synchronize()
    # canaries around the output stay untouched
    assert bool((buf[:offset_elems] == -7).all()) and bool((buf[offset_elems + n:] == -7).all())
    return to_numpy(out)


# (7, 4): under one 128-byte row (untiled); (9, 4), (65, 8), (3, 40): full rows
# plus a partial row; (2, 16): exactly one row; (3, 40): 5 runs per stream.
# One run per stream over whole rows (the tiled kernel's specialised form):
# (64, 4), (1000, 8), (100, 16), (513, 32) with runs of 1, 2, 4 and 8 groups.
SHAPES = [(1, 1), (3, 5), (257, 4), (100, 16), (33, 67), (1000, 8), (5, 130), (77, 96), (300, 48), (513, 32),
          (7, 4), (9, 4), (2, 16), (65, 8), (3, 40), (64, 4)]


@pytest.mark.parametrize("gen", GENS)
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("shape", SHAPES)
def test_fill_small_shapes(torch_cuda, orc, gen, dtype, shape):
    n_streams, dps = shape
    for seed, counter in [(0x5EED, 0), (2**64 - 1, 0xFFFFFFFF)]:
        ref = orc.fill(gen, dtype, seed, counter, n_streams, dps)
        got = gpu_fill(torch_cuda, gen, dtype, seed, counter, n_streams, dps)
        compare(dtype, got, ref)


@pytest.mark.parametrize("gen", GENS)
@pytest.mark.parametrize("dtype", DTYPES)
def test_fill_unaligned_output_takes_scalar_path(torch_cuda, orc, gen, dtype):
    # One element past a 16-byte boundary: element-aligned, not vector-aligned.
    ref = orc.fill(gen, dtype, 99, 3, 300, 16)
    got = gpu_fill(torch_cuda, gen, dtype, 99, 3, 300, 16, offset_elems=1)
    compare(dtype, got, ref)


@pytest.mark.parametrize("gen", GENS)
@pytest.mark.parametrize("dtype", DTYPES)
def test_fill_output_off_row_boundary(torch_cuda, orc, gen, dtype):
    # 16 bytes past an allocation's start: vector-aligned but not on a
    # 128-byte row, so the tensor store's rows straddle the allocation's.
    off = 2 if dtype == W.F64_UNIFORM else 4
    for shape in [(300, 16), (1000, 8), (41, 32)]:
        ref = orc.fill(gen, dtype, 1234, 5, *shape)
        got = gpu_fill(torch_cuda, gen, dtype, 1234, 5, *shape, offset_elems=off)
        compare(dtype, got, ref)


@pytest.mark.parametrize("dtype", [W.U32, W.F32_UNIFORM])
def test_fill_small_workload_full(torch_cuda, orc, dtype):
    c = W.FILL_SMALL
    ref = orc.fill(W.PHILOX, dtype, c["seed"], c["counter"], c["n_streams"], c["dps"], threads=8)
    got = gpu_fill(torch_cuda, W.PHILOX, dtype, c["seed"], c["counter"], c["n_streams"], c["dps"])
    compare(dtype, got, ref)


def test_fill_typed_entry_points_agree(torch_cuda):
    torch = torch_cuda
    s = torch.cuda.current_stream().cuda_stream
    for dtype, fn in [(W.U32, orand.orand_fill_u32), (W.F32_UNIFORM, orand.orand_fill_uniform_f32),
                      (W.F64_UNIFORM, orand.orand_fill_uniform_f64), (W.F32_NORMAL, orand.orand_fill_normal_f32)]:
        a = torch.empty(4096, dtype=orand.torch_dtype(dtype), device="cuda")
        b = torch.empty_like(a)
        fn(W.THREEFRY, 5, 6, 64, 64, a.data_ptr(), s)
        orand.orand_fill(W.THREEFRY, dtype, 5, 6, 64, 64, b.data_ptr(), s)
        torch.cuda.synchronize()
        assert torch.equal(a, b)


def test_fill_is_independent_of_stream_range_split(torch_cuda):
    # Streams [s0, s0 + n) with s0 a multiple of a power of two >= n are the
    # streams 0..n-1 of seed ^ s0 (key64 = seed ^ s): how ranks shard a fill.
    torch = torch_cuda
    seed, n = 0x5EED, 1 << 10
    full = orand.fill(W.SQUARES, W.U32, seed, 0, 4 * n, 16)
    for r in range(4):
        part = orand.fill(W.SQUARES, W.U32, seed ^ (r * n), 0, n, 16)
        assert torch.equal(full[r * n * 16:(r + 1) * n * 16], part)


@pytest.mark.parametrize("gen", GENS)
@pytest.mark.parametrize("dtype", DTYPES)
def test_fill_large_workload_every_value(torch_cuda, orc, gen, dtype):
    """The benchmark's 2^24 x 16 fill (2^28 values) in its launch
    configuration, compared with the oracle on every value: the oracle runs
    on all host threads over chunks of 2^21 streams.  Plus range and moments
    over the whole array."""
    import os

    torch = torch_cuda
    c = W.FILL_LARGE
    n_streams, dps = c["n_streams"], c["dps"]
    out = orand.fill(gen, dtype, c["seed"], c["counter"], n_streams, dps)
    torch.cuda.synchronize()
    host = to_numpy(out)
    threads = os.cpu_count() or 1
    chunk = 1 << 21
    for s0 in range(0, n_streams, chunk):
        ref = orc.fill(gen, dtype, c["seed"], c["counter"], chunk, dps, s_first=s0, threads=threads)
        compare(dtype, host[s0 * dps:(s0 + chunk) * dps], ref)
    del host, ref
    n = out.numel()
    if dtype == W.F32_UNIFORM:
        assert out.min().item() >= 0.0 and out.max().item() <= 1.0 - 2.0 ** -24
    if dtype in (W.F32_UNIFORM, W.F64_UNIFORM):
        x = out.double()
        assert abs(x.mean().item() - 0.5) < 5 * math.sqrt(1 / 12 / n)
        assert out.max().item() < 1.0
    if dtype == W.F32_NORMAL:
        x = out.double()
        assert x.abs().max().item() <= 5.7682
        assert abs(x.mean().item()) < 5 / math.sqrt(n)
        assert abs(x.var().item() - 1) < 5 * math.sqrt(2 / n)
    if dtype == W.U32:
        w = out.view(torch.int32)
        top = ((w >> 24) & 0xFF).bincount(minlength=256).double()
        chi2 = ((top - n / 256) ** 2 / (n / 256)).sum().item()
        assert abs(chi2 - 255) < 5 * math.sqrt(2 * 255)
    del out
    torch.cuda.empty_cache()


@pytest.mark.parametrize("gen", GENS)
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("shape", [(1000, 16), (101, 5)])
def test_fill_stream_ranges_concatenate(torch_cuda, orc, gen, dtype, shape):
    """orand_fill_streams: uneven, single-stream and empty ranges of one fill
    (tiled and untiled paths) concatenate to the whole fill, and a range far
    from stream 0 matches the oracle's streams there."""
    torch = torch_cuda
    n_streams, dps = shape
    full = orand.fill(gen, dtype, 0x5EED, 3, n_streams, dps)
    parts = torch.zeros_like(full)
    cuts = [0, 1, n_streams // 3, n_streams // 3, n_streams - 1, n_streams]
    for a, b in zip(cuts[:-1], cuts[1:]):
        if b > a:
            orand.fill(gen, dtype, 0x5EED, 3, b - a, dps, out=parts[a * dps:b * dps], first_stream=a)
    torch.cuda.synchronize()
    assert np.array_equal(to_numpy(parts), to_numpy(full))
    first = 2**40 + 12345
    got = to_numpy(orand.fill(gen, dtype, 0x5EED, 3, 300, dps, first_stream=first))
    compare(dtype, got, orc.fill(gen, dtype, 0x5EED, 3, 300, dps, s_first=first))


@pytest.mark.parametrize("extra", [9, 16])
def test_fill_over_2p30_rows_splits_launches(torch_cuda, orc, extra):
    """A u32 fill of 2^31 + extra streams x 16 words (128 GiB + 64 B per extra
    stream): more than the 2^30 128-byte rows one tensor-store launch
    addresses, so the tiled path runs a second launch of the extra streams,
    starting at stream 2^31.  With 9 its last 4 chunks form a partial row;
    with 16 it is whole rows, which the specialised kernel serves.  Exact on
    the streams around the split and the end, and on sampled streams."""
    torch = torch_cuda
    n_streams, dps, seed = (1 << 31) + extra, 16, 0x5EED
    torch.cuda.empty_cache()                   # return blocks cached by earlier tests
    free, _ = torch.cuda.mem_get_info()
    need = n_streams * dps * 4
    if free < need + (8 << 30):
        pytest.skip("needs %d GiB of free device memory" % ((need >> 30) + 8))
    out = torch.empty(n_streams * dps + 4, dtype=torch.int32, device="cuda")
    out[-4:] = -7
    orand.fill(W.PHILOX, W.U32, seed, 0, n_streams, dps, out=out[:n_streams * dps])
    torch.cuda.synchronize()
    assert bool((out[-4:] == -7).all())
    rng = np.random.default_rng(31)
    streams = np.unique(np.concatenate([
        [0, 1], np.arange((1 << 31) - 3, n_streams), rng.integers(0, n_streams, 64)]))
    idx = torch.as_tensor((streams[:, None] * dps + np.arange(dps)[None, :]).ravel(), device="cuda")
    got = to_numpy(out[idx]).reshape(len(streams), dps)
    for i, s in enumerate(streams):
        ref = orc.fill(W.PHILOX, W.U32, seed, 0, 1, dps, s_first=int(s))
        assert np.array_equal(got[i], ref), int(s)
    del out, idx
    torch.cuda.empty_cache()


def test_fills_on_concurrent_streams(torch_cuda, orc):
    """Fills of every generator enqueued on four streams at once (each call
    builds its own tensor map): every output equals the oracle."""
    torch = torch_cuda
    shape = (1000, 8)
    streams = [torch.cuda.Stream() for _ in range(4)]
    outs = []
    for rep in range(3):
        for gen, s in zip(GENS, streams):
            out = torch.empty(shape[0] * shape[1], dtype=torch.int32, device="cuda")
            orand.fill(gen, W.U32, 77 + rep, rep, *shape, out=out, stream=s)
            outs.append((gen, rep, out))
    torch.cuda.synchronize()
    for gen, rep, out in outs:
        assert np.array_equal(to_numpy(out), orc.fill(gen, W.U32, 77 + rep, rep, *shape)), (gen, rep)


def test_fill_captured_in_a_cuda_graph(torch_cuda, orc):
    """A tiled fill captured in a CUDA graph (its tensor map is a kernel
    parameter, copied at capture) replays to the same bits."""
    torch = torch_cuda
    shape = (300, 16)
    out = torch.zeros(shape[0] * shape[1], dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        orand.fill(W.PHILOX, W.U32, 5, 9, *shape, out=out, stream=s)   # configure outside the capture
    torch.cuda.synchronize()
    out.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        orand.fill(W.PHILOX, W.U32, 5, 9, *shape, out=out, stream=s)
    out.zero_()
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(to_numpy(out), orc.fill(W.PHILOX, W.U32, 5, 9, *shape))

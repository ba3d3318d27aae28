"""GPU parity of the ragged batcher.

Each request must equal the oracle's single-stream fill (gen, seed, counter,
length): bit-exact for u32 and uniforms, <= 4 ulp for normals.  The batch
is also compared with the one-launch-per-request baseline and across every
batcher configuration (the autotuner must never change bits).  Bytes
outside the requested ranges stay untouched.
"""
import os

import numpy as np
import pytest

from helpers import ulp_distance_f32

import paper_2310_19925_b300 as orand
from paper_2310_19925_b300 import workloads as W

pytestmark = pytest.mark.gpu

NP_DT = {W.U32: np.uint32, W.F32_UNIFORM: np.float32, W.F64_UNIFORM: np.float64, W.F32_NORMAL: np.float32}


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def mixed_requests(n, max_log2, seed, unaligned_every=7):
    """All generators and dtypes, log-uniform lengths, some offsets off the 16-byte grid."""
    recs, _ = W.ragged_requests(n, max_log2, list_seed=seed, dtypes=(0, 1, 2, 3))
    off = 0
    for i in range(n):
        e = W.ELEM_BYTES[int(recs[i]["dtype"])]
        off = (off + 15) // 16 * 16
        if i % unaligned_every == 3:
            off += e          # element-aligned, not 16-byte aligned
        recs[i]["out_offset_bytes"] = off
        off += int(recs[i]["length"]) * e
    return recs, off + 64


def request_values(host_bytes, r):
    dt = int(r["dtype"])
    o, L = int(r["out_offset_bytes"]), int(r["length"])
    return host_bytes[o:o + L * W.ELEM_BYTES[dt]].view(NP_DT[dt])


def check_request(orc, host_bytes, r):
    dt = int(r["dtype"])
    got = request_values(host_bytes, r)
    ref = orc.fill(int(r["gen"]), dt, int(r["seed"]), int(r["counter"]), 1, int(r["length"]))
    if dt == W.F32_NORMAL:
        assert ulp_distance_f32(got, ref).max(initial=0) <= 4
    elif dt == W.F32_UNIFORM:
        assert np.array_equal(got.astype(np.float64), ref)
    else:
        assert np.array_equal(got, ref)


def covered_mask(recs, nbytes):
    m = np.zeros(nbytes, bool)
    for r in recs:
        o = int(r["out_offset_bytes"])
        m[o:o + int(r["length"]) * W.ELEM_BYTES[int(r["dtype"])]] = True
    return m


def test_ragged_small_mixed_batch(torch_cuda, orc):
    recs, nbytes = mixed_requests(400, 12, seed=1)
    out = torch_cuda.zeros(nbytes, dtype=torch_cuda.uint8, device="cuda")
    orand.fill_ragged(recs, out=out)
    host = out.cpu().numpy()
    for r in recs:
        check_request(orc, host, r)
    assert not host[~covered_mask(recs, nbytes)].any()   # padding untouched


CONFIGS = [(64, 128, 4, 0), (128, 4096, 8, 1), (256, 8192, 16, 0), (512, 65536, 16, 2), (1024, 2048, 8, 0),
           (256, 132, 4, 3)]


def test_ragged_configs_do_not_change_bits(torch_cuda):
    torch = torch_cuda
    ctx = orand.Context()
    try:
        recs, nbytes = mixed_requests(300, 14, seed=2)
        ref = orand.fill_ragged(recs, out_bytes=nbytes, serial=True)
        for cfg in CONFIGS:
            orand.orand_ragged_set_config(ctx.handle, orand.RaggedConfig(*cfg))
            out = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
            orand.fill_ragged(recs, out=out, ctx=ctx)
            torch.cuda.synchronize()
            assert torch.equal(out, ref), cfg
            got = orand.orand_ragged_get_config(ctx.handle)
            assert (got.block, got.chunk_values, got.store_bytes, got.ctas_per_sm) == cfg
    finally:
        ctx.close()


def test_ragged_autotune_and_graph_reuse(torch_cuda):
    torch = torch_cuda
    ctx = orand.Context()
    try:
        recs, nbytes = mixed_requests(200, 13, seed=3)
        out = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
        orand.fill_ragged(recs, out=out, ctx=ctx)
        s1 = orand.orand_ragged_stats(ctx.handle)
        assert s1.tune_runs > 0 and s1.tuned_classes == 1 and s1.graph_builds == 1
        first = out.clone()
        # Same shape, new contents (other seeds): the tuned class and the graph are reused.
        recs2 = recs.copy()
        recs2["seed"] += 1000
        out2 = torch.zeros_like(out)
        orand.fill_ragged(recs2, out=out2, ctx=ctx)
        orand.fill_ragged(recs, out=out, ctx=ctx)
        torch.cuda.synchronize()
        s2 = orand.orand_ragged_stats(ctx.handle)
        assert s2.tune_runs == s1.tune_runs and s2.graph_builds == 1 and s2.graph_launches == 3
        assert torch.equal(out, first) and not torch.equal(out2, first)
        assert torch.equal(out2, orand.fill_ragged(recs2, out_bytes=nbytes, serial=True))
        # Another stream: the batch still orders after the previous one on this ctx.
        s = torch.cuda.Stream()
        out3 = torch.zeros_like(out)
        orand.fill_ragged(recs, out=out3, ctx=ctx, stream=s)
        s.synchronize()
        assert torch.equal(out3, first)
    finally:
        ctx.close()


def test_ragged_overlap_check(torch_cuda, monkeypatch):
    recs, nbytes = mixed_requests(10, 6, seed=4)
    recs[5]["out_offset_bytes"] = recs[4]["out_offset_bytes"]
    monkeypatch.setenv("ORAND_CHECK_OVERLAP", "1")
    with pytest.raises(orand.OrandError):
        orand.fill_ragged(recs, out_bytes=nbytes)


def test_ragged_extreme_keys_and_counters(torch_cuda, orc):
    """Every generator and dtype with seeds 0 and 2^64 - 1, counters 0 and
    2^32 - 1, and lengths around the group and chunk sizes."""
    recs = []
    for gen in (W.PHILOX, W.THREEFRY, W.SQUARES, W.TYCHE):
        for dt in (W.U32, W.F32_UNIFORM, W.F64_UNIFORM, W.F32_NORMAL):
            for seed, counter in [(0, 0), (2**64 - 1, 0xFFFFFFFF), (12345, 0xFFFFFFFF)]:
                for length in (1, 3, 17, 4096 + 5):
                    recs.append((gen, dt, seed, counter, 0, length, 0))
    recs = np.array(recs, dtype=W.REQUEST_DTYPE)
    off = 0
    for r in recs:
        off = (off + 15) // 16 * 16
        r["out_offset_bytes"] = off
        off += int(r["length"]) * W.ELEM_BYTES[int(r["dtype"])]
    out = orand.fill_ragged(recs, out_bytes=off + 16)
    host = out.cpu().numpy()
    for r in recs:
        check_request(orc, host, r)


def test_ragged_empty_and_zero_length(torch_cuda, orc):
    recs, nbytes = mixed_requests(20, 5, seed=5)
    recs["length"][::3] = 0
    out = orand.fill_ragged(recs, out_bytes=nbytes)
    host = out.cpu().numpy()
    for r in recs:
        if r["length"]:
            check_request(orc, host, r)
    assert not host[~covered_mask(recs, nbytes)].any()


def test_ragged_full_workload_every_request(torch_cuda, orc):
    """100,000 requests, lengths log-uniform in [1, 2^20], ~30 GB of output,
    one graph-launched persistent kernel; every request compared with the
    oracle (7.49e9 values), which runs on all host threads, longest requests
    first, over slices of at most 2 GiB of the output; and the
    one-launch-per-request baseline writes the same bytes on a subset."""
    import os
    from concurrent.futures import ThreadPoolExecutor

    torch = torch_cuda
    recs, total = W.ragged_requests()
    out = torch.zeros(total, dtype=torch.uint8, device="cuda")
    orand.fill_ragged(recs, out=out)
    torch.cuda.synchronize()
    elem = np.where(recs["dtype"] == W.F64_UNIFORM, 8, 4).astype(np.uint64)
    ends = (recs["out_offset_bytes"] + recs["length"] * elem).astype(np.int64)
    starts = recs["out_offset_bytes"].astype(np.int64)
    n, i, checked = len(recs), 0, 0
    with ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        while i < n:
            j = max(i + 1, int(np.searchsorted(ends, starts[i] + (2 << 30), side="right")))
            host = out[int(starts[i]):int(ends[j - 1])].cpu().numpy()
            sub = recs[i:j].copy()
            sub["out_offset_bytes"] -= np.uint64(starts[i])
            order = np.argsort(-sub["length"].astype(np.int64))
            for _ in ex.map(lambda k: check_request(orc, host, sub[k]), order):
                checked += 1
            i = j
    assert checked == n
    # The per-request baseline writes the same bytes on a subset.
    sub = recs[:1500].copy()
    end = int(sub["out_offset_bytes"][-1] + sub["length"][-1] * 4)
    base = orand.fill_ragged(sub, out_bytes=end, serial=True)
    torch.cuda.synchronize()
    assert torch.equal(base, out[:end])
    del out
    torch.cuda.empty_cache()

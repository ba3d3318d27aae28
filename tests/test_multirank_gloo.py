"""Multi-rank sharding on CPU: two gloo ranks, no GPU.

The hot path shards without a data-path collective: a fill splits its stream
range, and a walk its particle range, across ranks.  Only the walk's loss and
gradients need a sum over ranks.  These tests run the sharding arithmetic
used by bench.py on the CPU oracle, in world-size-2 gloo process groups.
  * A power-of-two stream block [r*n, (r+1)*n) is the fill with seed ^ (r*n).
  * Particle ranges use p_first = r*n with the global particle count as the
    loss normaliser.  All-reducing the per-rank sums then reproduces the
    unsharded loss and gradients.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    import oracle

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # Fill: rank r owns streams [r*n, (r+1)*n) of the global problem.
        n, dps, seed = 64, 8, 0x5EED
        part = oracle.fill(0, 3, seed ^ (rank * n), 0, n, dps)
        parts = [None] * world
        dist.all_gather_object(parts, part)
        # Walk: rank r owns particles [r*m, (r+1)*m); gradients are sums.
        m, steps, P = 40, 30, 40 * world
        dt = float(np.float32(1e-3))
        mu = (0.1, -0.2, 0.05)
        xT, _ = oracle.walk3d_forward(0, m, steps, 8, dt, mu, 0.5, p_first=rank * m)
        loss = oracle.walk3d_loss(xT, 2.0, P)
        dmu, dsig, _ = oracle.walk3d_adjoint(0, m, steps, dt, xT, 2.0, P, p_first=rank * m)
        t = torch.tensor([loss, dmu[0], dmu[1], dmu[2], dsig], dtype=torch.float64)
        dist.all_reduce(t)
        q.put((rank, np.concatenate(parts), t.numpy()))
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_matches_unsharded(orc):
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    full_fill = orc.fill(0, 3, 0x5EED, 0, 64 * world, 8)
    m, steps, P = 40, 30, 40 * world
    dt = float(np.float32(1e-3))
    xT, _ = orc.walk3d_forward(0, P, steps, 8, dt, (0.1, -0.2, 0.05), 0.5)
    loss = orc.walk3d_loss(xT, 2.0, P)
    dmu, dsig, _ = orc.walk3d_adjoint(0, P, steps, dt, xT, 2.0, P)
    want = np.array([loss, *dmu, dsig])
    for rank, fill, red in res:
        assert np.array_equal(fill, full_fill)
        assert np.allclose(red, want, rtol=1e-12, atol=0)


def _stream_worker(rank, world, port, q):
    """The parallel-stream battery sharded by iteration range: rank r counts
    the micro-streams of iterations [r*I, (r+1)*I) and the counts are summed
    over ranks."""
    import torch
    import torch.distributed as dist

    from oracle import stream_stats as S

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n_part, draws, iters = 200, 3, 32                  # 32 iterations: whole birthday samples
        w = S.micro_stream_words(0, 0, n_part, draws, rank * iters, iters)
        tup = S.tuple_counts(w, 3, 4, 28, 3).astype(np.int64)
        bday = S.birthday_counts(w, 6, 16, 0, 40).astype(np.int64)
        gaps, _ = S.gap_counts(w, 0, 1 << 28, 64)
        t = torch.from_numpy(np.concatenate([tup, bday, gaps.astype(np.int64)]))
        dist.all_reduce(t)
        q.put((rank, t.numpy()))
    finally:
        dist.destroy_process_group()


def test_two_rank_stream_battery_matches_one_stream():
    """Summed over ranks, tuple and birthday counts equal those of the whole
    stream (each rank's share is a multiple of 32 iterations, so no tuple or
    sample straddles a rank boundary); the gap counts miss exactly the gap
    that spans each rank boundary."""
    from oracle import stream_stats as S

    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_stream_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = S.micro_stream_words(0, 0, 200, 3, 0, 32 * world)
    tup = S.tuple_counts(w, 3, 4, 28, 3).astype(np.int64)
    bday = S.birthday_counts(w, 6, 16, 0, 40).astype(np.int64)
    gaps, _ = S.gap_counts(w, 0, 1 << 28, 64)
    nt, nb = tup.size, bday.size
    for rank, red in res:
        assert np.array_equal(red[:nt], tup)
        assert np.array_equal(red[nt:nt + nb], bday)
        assert int(gaps.astype(np.int64).sum() - red[nt + nb:].sum()) == world - 1

"""Multi-rank sharding on CPU: world-size-2 and -3 gloo ranks, no GPU.

The hot path shards without a data-path collective: a fill splits its stream
range, a ragged batch its request list, and a walk its particle range
across ranks.  Only the walk's loss and gradients need a sum over ranks.
These tests drive the product's sharding helpers
(paper_2310_19925_b300.shard: split_range, ragged_shard,
allreduce_walk_scalars) with per-rank partials computed by the CPU oracle:
  * uneven stream ranges of a fill concatenate to the unsharded fill;
  * every request of a ragged list is served by exactly one rank, with the
    unsharded values, and the Tyche chains are spread over the ranks;
  * particle ranges with the global particle count as the loss normaliser,
    all-reduced by the helper, reproduce the unsharded loss and gradients
    (constant drift, and OU drift with dL/dkappa).
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

FILL = dict(gen=1, dtype=3, seed=0x5EED, n_streams=101, dps=6)
WALK = dict(P=81, steps=30, K=8, mu=(0.1, -0.2, 0.05), sigma=0.5, kappa=1.5, k=2.0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _ragged_list():
    from paper_2310_19925_b300 import workloads as W

    return W.ragged_requests(60, 12, list_seed=7, dtypes=(0, 1, 2, 3))[0]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2310_19925_b300 import shard

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # Fill: this rank's stream range of the global problem.
        f = FILL
        first, count = shard.split_range(f["n_streams"], rank, world)
        part = oracle.fill(f["gen"], f["dtype"], f["seed"], 0, count, f["dps"], s_first=first)
        fills = [None] * world
        dist.all_gather_object(fills, (first, part))
        # Ragged: this rank's requests, re-packed for a buffer of its own.
        mine, total, idx = shard.ragged_shard(_ragged_list(), rank, world)
        vals = oracle.ragged(mine)
        assert total >= sum(int(r["length"]) for r in mine)
        rag = [None] * world
        dist.all_gather_object(rag, (idx, vals))
        # Walks: this rank's particles, normalised by the global count.
        w = WALK
        dt = float(np.float32(1e-3))
        p_first, m = shard.split_range(w["P"], rank, world)
        xT, _ = oracle.walk3d_forward(0, m, w["steps"], w["K"], dt, w["mu"], w["sigma"], p_first=p_first)
        dmu, dsig, _ = oracle.walk3d_adjoint(0, m, w["steps"], dt, xT, w["k"], w["P"], p_first=p_first)
        t_loss = torch.tensor(oracle.walk3d_loss(xT, w["k"], w["P"]), dtype=torch.float64)
        t_dmu = torch.tensor(dmu, dtype=torch.float64)
        t_dsig = torch.tensor(dsig, dtype=torch.float64)
        shard.allreduce_walk_scalars(t_loss, t_dmu, t_dsig)
        oxT, _, xs = oracle.walk3d_ou_forward(0, m, w["steps"], w["K"], dt, w["mu"], w["sigma"], w["kappa"],
                                              p_first=p_first)
        odmu, odsig, odk, _ = oracle.walk3d_ou_adjoint(0, m, w["steps"], dt, w["kappa"], xs, w["k"], w["P"],
                                                       p_first=p_first)
        o_loss = torch.tensor(oracle.walk3d_loss(oxT, w["k"], w["P"]), dtype=torch.float64)
        o_dmu = torch.tensor(odmu, dtype=torch.float64)
        o_dsig = torch.tensor(odsig, dtype=torch.float64)
        o_dk = torch.tensor(odk, dtype=torch.float64)
        shard.allreduce_walk_scalars(o_loss, o_dmu, o_dsig, o_dk)
        walk = np.array([t_loss.item(), *t_dmu.tolist(), t_dsig.item()])
        ou = np.array([o_loss.item(), *o_dmu.tolist(), o_dsig.item(), o_dk.item()])
        q.put((rank, fills, rag, walk, ou))
    finally:
        dist.destroy_process_group()


def _run(target, world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


@pytest.mark.parametrize("world", [2, 3])
def test_sharding_helpers_reproduce_the_unsharded_problem(orc, world):
    res = _run(_worker, world)
    f, w = FILL, WALK
    full_fill = orc.fill(f["gen"], f["dtype"], f["seed"], 0, f["n_streams"], f["dps"])
    recs = _ragged_list()
    full_rag = orc.ragged(recs)
    dt = float(np.float32(1e-3))
    xT, _ = orc.walk3d_forward(0, w["P"], w["steps"], w["K"], dt, w["mu"], w["sigma"])
    dmu, dsig, _ = orc.walk3d_adjoint(0, w["P"], w["steps"], dt, xT, w["k"], w["P"])
    want = np.array([orc.walk3d_loss(xT, w["k"], w["P"]), *dmu, dsig])
    oxT, _, xs = orc.walk3d_ou_forward(0, w["P"], w["steps"], w["K"], dt, w["mu"], w["sigma"], w["kappa"])
    odmu, odsig, odk, _ = orc.walk3d_ou_adjoint(0, w["P"], w["steps"], dt, w["kappa"], xs, w["k"], w["P"])
    want_ou = np.array([orc.walk3d_loss(oxT, w["k"], w["P"]), *odmu, odsig, odk])
    for rank, fills, rag, walk, ou in res:
        fills = sorted(fills, key=lambda t: t[0])
        assert np.array_equal(np.concatenate([p for _, p in fills]), full_fill)
        seen = np.concatenate([idx for idx, _ in rag])
        assert np.array_equal(np.sort(seen), np.arange(len(recs)))       # every request, once
        for idx, vals in rag:
            for i, v in zip(idx, vals):
                assert np.array_equal(v, full_rag[i]), int(i)
        assert np.allclose(walk, want, rtol=1e-12, atol=0)
        assert np.allclose(ou, want_ou, rtol=1e-12, atol=0)


def test_split_range_and_ragged_partition_on_the_host():
    from paper_2310_19925_b300 import shard
    from paper_2310_19925_b300 import workloads as W

    for n in (0, 1, 7, 100, 2**40 + 3):
        for world in (1, 2, 3, 8):
            spans = [shard.split_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and sum(c for _, c in spans) == n
            assert all(a + c == b for (a, c), (b, _) in zip(spans, spans[1:]))
            assert max(c for _, c in spans) - min(c for _, c in spans) <= 1
    recs, _ = W.ragged_requests(4000, 20, list_seed=3)
    parts = shard.ragged_partition(recs, 4)
    assert np.array_equal(np.sort(np.concatenate(parts)), np.arange(len(recs)))
    ty = recs["gen"] == W.TYCHE
    longest = np.argsort(-recs["length"][ty].astype(np.int64))[:4]
    owners = {r for r, p in enumerate(parts) for i in np.nonzero(ty)[0][longest] if i in set(p.tolist())}
    assert len(owners) == 4                                            # the four longest chains on four ranks
    nbytes = [int((recs["length"][p] * np.where(recs["dtype"][p] == 2, 8, 4)).sum()) for p in parts]
    assert max(nbytes) <= 1.05 * min(nbytes)                           # bytes balanced within 5 %
    with pytest.raises(ValueError):
        shard.split_range(10, 3, 3)


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
    res = _run(_stream_worker, world)
    w = S.micro_stream_words(0, 0, 200, 3, 0, 32 * world)
    tup = S.tuple_counts(w, 3, 4, 28, 3).astype(np.int64)
    bday = S.birthday_counts(w, 6, 16, 0, 40).astype(np.int64)
    gaps, _ = S.gap_counts(w, 0, 1 << 28, 64)
    nt, nb = tup.size, bday.size
    for rank, red in res:
        assert np.array_equal(red[:nt], tup)
        assert np.array_equal(red[nt:nt + nb], bday)
        assert int(gaps.astype(np.int64).sum() - red[nt + nb:].sum()) == world - 1

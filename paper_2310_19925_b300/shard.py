"""Sharding of the hot path across ranks (one process per GPU).

Every value the library produces is a fixed function of (generator, key,
counter, index) (§3 of the paper: a stream is named by a seed and a counter,
and streams are independent), so ranks split the work with no data exchange:

* fills split the stream range: rank r fills streams [first, first + count)
  of the whole problem with orand_fill_streams;
* walks split the particle range (p_first, with the global particle count
  as the loss normaliser p_total);
* ragged batches split the request list; each rank serves its share into a
  buffer of its own.

The one exchange is the walk's loss and gradients: each rank's values are
sums over its own particles divided by the global count, so one sum
all-reduce of five scalars (loss, dL/dmu x 3, dL/dsigma; dL/dkappa with the
OU drift) gives the whole problem's.  dL/dx0 stays with the rank that owns
the particles.

Host logic only; the all-reduce takes torch tensors and a torch.distributed
process group (gloo on CPU tensors, NCCL on CUDA tensors).
"""
from __future__ import annotations

import heapq

import numpy as np

from .workloads import ELEM_BYTES, REQUEST_DTYPE, TYCHE


def split_range(n_total: int, rank: int, world: int):
    """Contiguous share of [0, n_total) for `rank` of `world`: (first, count).
    The first n_total % world ranks get one item more; shares concatenate
    in rank order."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside a world of %d" % (rank, world))
    if n_total < 0:
        raise ValueError("negative size")
    base, extra = divmod(n_total, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def _request_bytes(recs):
    elem = np.array([ELEM_BYTES[d] for d in range(4)], np.uint64)[recs["dtype"]]
    return (recs["length"] * elem).astype(np.int64)


def ragged_partition(requests, world: int):
    """Split a ragged request list over `world` ranks: a list of index
    arrays, one per rank, each in ascending order.

    Two kinds of cost decide a rank's batch time: the bytes it writes (the
    random-access generators stream at HBM speed) and its longest Tyche
    request, which one GPU thread runs as a serial chain.  So Tyche requests
    are placed first, longest first, each on the rank with the least Tyche
    work so far (longest-processing-time order), which spreads the long
    chains; then the other requests, largest first, each on the rank with
    the fewest bytes so far, counting the Tyche requests' bytes too."""
    recs = np.ascontiguousarray(requests, dtype=REQUEST_DTYPE)
    if world < 1:
        raise ValueError("world must be >= 1")
    nbytes = _request_bytes(recs)
    tyche = recs["gen"] == TYCHE
    owner = np.empty(len(recs), np.int64)
    chain = [(0, r) for r in range(world)]                 # (Tyche words so far, rank)
    lengths = recs["length"].astype(np.int64)
    for i in sorted(np.nonzero(tyche)[0], key=lambda k: (-lengths[k], k)):
        load, r = heapq.heappop(chain)
        owner[i] = r
        heapq.heappush(chain, (load + int(lengths[i]), r))
    load_bytes = np.zeros(world, np.int64)
    for i in np.nonzero(tyche)[0]:
        load_bytes[owner[i]] += nbytes[i]
    heap = [(int(load_bytes[r]), r) for r in range(world)]
    heapq.heapify(heap)
    for i in sorted(np.nonzero(~tyche)[0], key=lambda k: (-nbytes[k], k)):
        load, r = heapq.heappop(heap)
        owner[i] = r
        heapq.heappush(heap, (load + int(nbytes[i]), r))
    return [np.nonzero(owner == r)[0] for r in range(world)]


def ragged_shard(requests, rank: int, world: int, align: int = 16):
    """This rank's share of a ragged request list, re-packed for a buffer of
    its own: (records, buffer bytes, global indices).  Records keep their
    generator, dtype, seed, counter and length (so their values are those of
    the unsharded batch); their output offsets are packed in index order,
    each start rounded up to `align` bytes."""
    recs = np.ascontiguousarray(requests, dtype=REQUEST_DTYPE)
    idx = ragged_partition(recs, world)[rank]
    mine = recs[idx].copy()
    nbytes = _request_bytes(mine)
    padded = (nbytes + (align - 1)) // align * align
    offs = np.zeros(len(mine), np.int64)
    if len(mine) > 1:
        offs[1:] = np.cumsum(padded[:-1])
    mine["out_offset_bytes"] = offs.astype(np.uint64)
    total = int(offs[-1] + padded[-1]) if len(mine) else 0
    return mine, total, idx


def allreduce_walk_scalars(loss, dmu=None, dsigma=None, dkappa=None, group=None):
    """Sum the walk's loss and scalar gradients over the ranks of `group`, in
    place, with one all-reduce.  Each argument is a torch tensor (0-dim, or
    (3,) for dmu) or None; with a per-rank p_total equal to the global
    particle count, the sums are the whole problem's values."""
    import torch
    import torch.distributed as dist

    parts = [t for t in (loss, dmu, dsigma, dkappa) if t is not None]
    if not parts or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return
    flat = torch.cat([t.detach().reshape(-1).to(torch.float64) for t in parts])
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    k = 0
    for t in parts:
        n = t.numel()
        t.copy_(flat[k:k + n].reshape(t.shape).to(t.dtype))
        k += n

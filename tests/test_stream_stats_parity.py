"""The parallel-stream harness on the GPU against the oracle.

Bars: the concatenated micro-stream is bit-exact; every count (tuples, gaps,
birthday spacings) is exact, since counts are integers.  The statistics are
checked on numpy PCG64 words copied to the device, so their inputs come
from neither side; ragged lengths, span and piece boundaries, empty inputs,
streams with no hit or only hits, and the parameter limits are covered.
At the paper's configuration (16,000 particles x 3 words, lengthened to
2^30 words) every generator runs the whole battery: the totals obey exact
identities, the first chunk's counts equal the oracle's, and every p-value
stays inside (1e-10, 1 - 1e-10).
"""
import numpy as np
import pytest

import paper_2310_19925_b300 as orand
from oracle import stream_stats as S
from paper_2310_19925_b300 import stream_tests as ST
from paper_2310_19925_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def dev_words(torch, w):
    return torch.from_numpy(np.asarray(w, np.uint32).view(np.int32).copy()).cuda()


def host_u32(t):
    return t.cpu().numpy().view(np.uint32)


def pcg(n, seed=1):
    return np.random.default_rng(seed).integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)


@pytest.mark.parametrize("gen", [W.PHILOX, W.THREEFRY, W.SQUARES, W.TYCHE])
@pytest.mark.parametrize("draws", [1, 3, 4, 7, 64])
def test_micro_streams_bit_exact(torch_cuda, orc, gen, draws):
    n_streams, c0, nc = 1000 + 7, 2**32 - 5, 5
    got = orand.fill_micro_streams(gen, 0x5EED, n_streams, draws, c0, nc)
    torch_cuda.cuda.synchronize()
    assert np.array_equal(host_u32(got), S.micro_stream_words(gen, 0x5EED, n_streams, draws, c0, nc))


@pytest.mark.parametrize("n,t,bits,shift,stride", [(100003, 1, 8, 24, 1), (100003, 1, 8, 0, 1),
                                                   (99999, 2, 6, 26, 2), (99999, 3, 4, 28, 3),
                                                   (77777, 4, 3, 1, 4), (5000, 1, 14, 18, 1),
                                                   (4099, 2, 7, 3, 1), (2, 3, 4, 28, 3), (3, 3, 4, 28, 3),
                                                   (3, 1, 8, 24, 1), (6, 1, 4, 0, 1)])
def test_tuples_exact(torch_cuda, n, t, bits, shift, stride):
    w = pcg(n)
    want = S.tuple_counts(w, t, bits, shift, stride) + S.tuple_counts(w[: n // 2], t, bits, shift, stride)
    # 16-byte-aligned words (the four-word loads of single-word tuples) and
    # words one element past that (one-word loads)
    padded = dev_words(torch_cuda, np.concatenate([np.zeros(1, np.uint32), w]))
    for words in (dev_words(torch_cuda, w), padded[1:]):
        c = orand.stat_tuples(words, t, bits, shift, stride)
        c = orand.stat_tuples(words[: n // 2], t, bits, shift, stride, counts=c)  # accumulates
        assert np.array_equal(c.cpu().numpy().astype(np.uint64), want)


@pytest.mark.parametrize("n,lo,hi,t_max", [(8192 * 3 + 77, 0, 1 << 28, 64), (100000, 3 << 30, 1 << 32, 8),
                                           (50000, 12345, 12345 + (1 << 20), 4096), (31, 0, 1 << 31, 1),
                                           (8192, 0, 1 << 32, 16)])
def test_gaps_exact(torch_cuda, n, lo, hi, t_max):
    w = pcg(n, 3)
    want, wcarry = S.gap_counts(w, lo, hi, t_max)
    # 16-byte-aligned words (four-word loads) and words one element past
    # that (one-word loads)
    padded = dev_words(torch_cuda, np.concatenate([np.zeros(1, np.uint32), w]))
    for words in (dev_words(torch_cuda, w), padded[1:]):
        c, carry = orand.stat_gaps(words, lo, hi, t_max)
        assert np.array_equal(c.cpu().numpy().astype(np.uint64), want)
        assert int(carry.item()) & (2**64 - 1) == (orand.GAP_NO_HIT if wcarry is None else wcarry)


def test_gaps_in_pieces_with_device_carry(torch_cuda):
    """Pieces fed in order, with gaps across span and piece boundaries, a
    long stretch without hits spanning whole spans and whole pieces."""
    w = pcg(200000, 5)
    lo, hi, t_max = 0, 1 << 26, 300
    w[20000:70000] |= np.uint32(1 << 31)          # 50,000 words with no hit
    cuts = [0, 1, 8192, 8193, 25000, 31000, 90000, 90001, 200000]
    c, carry = None, None
    for a, b in zip(cuts[:-1], cuts[1:]):
        c, carry = orand.stat_gaps(dev_words(torch_cuda, w[a:b]), lo, hi, t_max, counts=c, carry=carry)
    want, wcarry = S.gap_counts(w, lo, hi, t_max)
    assert np.array_equal(c.cpu().numpy().astype(np.uint64), want)
    assert int(carry.item()) == wcarry


def test_gaps_degenerate(torch_cuda):
    torch = torch_cuda
    z = np.zeros(30000, np.uint32)
    c, carry = orand.stat_gaps(dev_words(torch, z), 1, 2, 8)          # no hit at all
    assert int(c.sum().item()) == 0 and int(carry.item()) & (2**64 - 1) == orand.GAP_NO_HIT
    c, carry = orand.stat_gaps(dev_words(torch, z), 0, 1, 8)          # every word a hit
    assert c.cpu().numpy().tolist() == [29999] + [0] * 8 and int(carry.item()) == 0
    c, carry = orand.stat_gaps(torch.empty(0, dtype=torch.int32, device="cuda"), 0, 1, 8)   # empty
    assert int(c.sum().item()) == 0


@pytest.mark.parametrize("n,log2_n,bits,shift,r_max", [(4096 * 5 + 100, 12, 32, 0, 16), (4096 * 3, 12, 20, 12, 4096),
                                                       (64 * 50, 6, 10, 22, 40), (4 * 30 + 3, 2, 4, 0, 8),
                                                       (512 * 9, 9, 1, 31, 600), (1024 * 4, 10, 24, 8, 1)])
def test_birthday_exact(torch_cuda, n, log2_n, bits, shift, r_max):
    w = pcg(n, 7)
    c = orand.stat_birthday(dev_words(torch_cuda, w), log2_n, bits, shift, r_max)
    assert np.array_equal(c.cpu().numpy().astype(np.uint64), S.birthday_counts(w, log2_n, bits, shift, r_max))


def test_birthday_degenerate(torch_cuda):
    # all birthdays equal: spacings 0 (n-1 times) and m, so R = n - 2
    z = np.full(4096 * 2, 7, np.uint32)
    c = orand.stat_birthday(dev_words(torch_cuda, z), 12, 32, 0, 4096)
    assert c[4094].item() == 2 and int(c.sum().item()) == 2
    c = orand.stat_birthday(dev_words(torch_cuda, z[:4095]), 12, 32, 0, 16)   # no whole sample
    assert int(c.sum().item()) == 0


@pytest.mark.parametrize("gen", [W.PHILOX, W.THREEFRY, W.SQUARES, W.TYCHE])
def test_parallel_stream_battery_full(torch_cuda, orc, gen):
    """§5's configuration, 16,000 particles x 3 words, lengthened to 2^30
    words: exact totals, the first 32 iterations against the oracle, and
    no p-value outside (1e-10, 1 - 1e-10)."""
    res, timing = ST.run(gen, seed=0, n_words=1 << 30)
    n = timing["words"]
    assert n == (1 << 30) // 48000 * 48000
    for name, r in res.items():
        if r["kind"] == "tuples":
            assert r["samples"] == (n - r["t"]) // r["stride"] + 1
        elif r["kind"] == "birthday":
            assert r["samples"] == n >> r["log2_n"]
        assert r["verdict"] == "pass", (gen, name, r["p"])
    # the first chunk's counts equal the oracle's on the oracle's own words
    small, _ = ST.run(gen, seed=0, n_words=32 * 48000)
    w = S.micro_stream_words(gen, 0, 16000, 3, 0, 32)
    for name, kind, prm in ST.BATTERY:
        if kind == "tuples":
            want = S.tuple_counts(w, prm["t"], prm["bits"], prm["shift"], prm["stride"])
        elif kind == "gaps":
            want, _ = S.gap_counts(w, prm["lo"], prm["hi"], prm["t_max"])
        else:
            want = S.birthday_counts(w, prm["log2_n"], prm["bits"], prm["shift"], prm["r_max"])
        assert np.array_equal(small[name]["counts"], want), name


def test_battery_rejects_planted_correlation(torch_cuda):
    """Every particle drawing the same 3 words per iteration (the particle
    id dropped from the key): the GPU counts must fail the battery."""
    torch = torch_cuda
    one = orand.fill_micro_streams(W.PHILOX, 0x5EED, 1, 3, 0, 64)      # 64 iterations, one particle
    w = one.view(64, 1, 3).expand(64, 16000, 3).contiguous().view(-1)
    verdicts = {}
    for name, kind, prm in ST.BATTERY:
        if kind == "tuples":
            c = orand.stat_tuples(w, prm["t"], prm["bits"], prm["shift"], prm["stride"])
        elif kind == "gaps":
            c, _ = orand.stat_gaps(w, prm["lo"], prm["hi"], prm["t_max"])
        else:
            c = orand.stat_birthday(w, prm["log2_n"], prm["bits"], prm["shift"], prm["r_max"])
        verdicts[name] = ST.evaluate(kind, prm, c.cpu().numpy())["verdict"]
    assert verdicts["triples_hi4"] == "fail" and verdicts["birthday_4096_2p32"] == "fail"
    torch.cuda.synchronize()


def test_birthday_extreme_spacings(torch_cuda):
    """Spacings of exactly 2^32 - 1 (the largest 32-bit value) and 2^32 (the
    wrap spacing when all birthdays are equal), in 32-bit years."""
    M = 0xFFFFFFFF
    samples = [[0, M, M, M], [0, M, 0, M], [0, M, 5, 7], [M, M, M, M], [0, 1, 2, 3], [M, 0, 1, M - 1]]
    w = np.array([x for s in samples for x in s], np.uint32)
    c = orand.stat_birthday(dev_words(torch_cuda, w), 2, 32, 0, 8)
    assert np.array_equal(c.cpu().numpy().astype(np.uint64), S.birthday_counts(w, 2, 32, 0, 8))


def test_birthday_bucket_overflow_falls_back(torch_cuda):
    """A sample whose birthdays crowd into few buckets (only the low 12 bits
    vary) takes the bounded fallback sort; counts still equal the oracle's."""
    rng = np.random.default_rng(8)
    w = (rng.integers(0, 4096, size=4096 * 6, dtype=np.uint64).astype(np.uint32) | np.uint32(0x5A5A0000))
    c = orand.stat_birthday(dev_words(torch_cuda, w), 12, 32, 0, 4096)
    assert np.array_equal(c.cpu().numpy().astype(np.uint64), S.birthday_counts(w, 12, 32, 0, 4096))


def test_birthday_colliding_and_repeated_spacings(torch_cuda):
    """Samples whose spacings take few values, all of which share one slot of
    the kernel's multiplicative hash (the 4n-slot table of n = 4096), so the
    distinct spacings are resolved one round at a time and most spacings are
    repeats.  Counts equal the oracle's."""
    rng = np.random.default_rng(11)
    v = np.arange(1, 1 << 19, dtype=np.uint64)
    slot = ((v * np.uint64(0x9E3779B1)) & np.uint64(0xFFFFFFFF)) >> np.uint64(32 - 14)
    target = np.bincount(slot.astype(np.int64)).argmax()
    vals = v[slot == target]                                  # distinct values, one slot
    assert len(vals) >= 24
    samples = []
    for kinds in (len(vals), 8, 1):
        sp = rng.choice(vals[:kinds], size=4095)
        keys = np.concatenate([[0], np.cumsum(sp)]).astype(np.uint64) + np.uint64(rng.integers(0, 1 << 20))
        assert keys[-1] < (1 << 32)
        samples.append(rng.permutation(keys.astype(np.uint32)))
    w = np.concatenate(samples)
    c = orand.stat_birthday(dev_words(torch_cuda, w), 12, 32, 0, 4096)
    assert np.array_equal(c.cpu().numpy().astype(np.uint64), S.birthday_counts(w, 12, 32, 0, 4096))
